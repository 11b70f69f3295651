// Shared definitions of the CUDA side of libhuff (kernels and C ABI layer).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "huff.h"

namespace huff {

constexpr uint32_t kHeaderBytes = HUFF_HEADER_BYTES;
constexpr uint32_t kMaxCodeLen = HUFF_MAX_CODE_LEN;

// Bounded spin: number of polls before a device wait gives up with
// HUFF_ERR_TIMEOUT.  Each poll is an L2 round trip (~1 us with the back-off),
// so the limit is a few seconds of wall time.
constexpr uint32_t kSpinLimit = 1u << 22;

// ---- status word: "first error wins", read by every kernel first ----------
__device__ __forceinline__ void set_status(int32_t *st, int32_t code)
{
    if (st)
        atomicCAS(st, 0, code);
}

__device__ __forceinline__ bool chain_failed(const int32_t *st)
{
    return st && *reinterpret_cast<const volatile int32_t *>(st) != 0;
}

// ---- streaming loads / stores ---------------------------------------------
__device__ __forceinline__ uint4 ld_stream16(const void *p)
{
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ uint64_t ld_volatile_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_volatile_u64(unsigned long long *p, uint64_t v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"((unsigned long long)v)
                 : "memory");
}

// ---- stream header access (device; GB300 is little-endian) ----------------
struct StreamHeader {
    uint64_t n;
    uint32_t chunk_symbols;
    uint32_t max_len;
};

__host__ __device__ __forceinline__ bool chunk_symbols_valid(uint32_t cs)
{
    return cs >= HUFF_MIN_CHUNK_SYMBOLS && cs <= HUFF_MAX_CHUNK_SYMBOLS && (cs % 16u) == 0;
}

__host__ __device__ __forceinline__ uint64_t ceil_div_u64(uint64_t a, uint64_t b)
{
    return a / b + (a % b != 0);
}

// Launch helpers defined in api.cu.
int device_sm_count();

}  // namespace huff

// Kernel launchers (one per translation unit); each returns a cudaError_t.
namespace huff {
cudaError_t launch_histogram(const uint8_t *d_in, uint64_t n, unsigned long long *d_hist,
                             cudaStream_t s);
cudaError_t launch_build_codebook(const unsigned long long *d_hist, huff_codebook_t *d_cb,
                                  int32_t *d_status, cudaStream_t s);
cudaError_t launch_encode(const uint8_t *d_in, uint64_t n, const huff_codebook_t *d_cb,
                          uint32_t cs, uint8_t *d_out, uint64_t out_cap,
                          unsigned long long *d_out_bytes, void *d_ws, int32_t *d_status,
                          cudaStream_t s);
cudaError_t launch_decode(const uint8_t *d_stream, uint64_t bytes, uint8_t *d_out,
                          uint64_t out_cap, unsigned long long *d_n, int32_t *d_status,
                          cudaStream_t s);
uint64_t encode_workspace_bytes(uint64_t n);
}  // namespace huff
