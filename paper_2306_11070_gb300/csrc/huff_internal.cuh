// Shared definitions of the CUDA side of libhuff (kernels and C ABI layer).
#pragma once

#include <atomic>
#include <cstdint>
#include <mutex>

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

// ---- shared-memory addresses ----------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---- integer arithmetic on the FMA pipe, shared-memory access by address --
// Integer constants read from the constant bank.  A multiply by one of them
// is an IMAD, which runs on the FMA pipe; adds, conditional adds and
// constant shifts written that way leave the ALU pipe (which executes the
// shifts, logic ops and compares, at half a warp per cycle) to the work only
// it can do.  The values are not visible to the compiler, so it cannot turn
// the multiplies back into shifts and adds.
enum { kOne, kMinus1, kFour, kEight, k32, kMinus32, k128, kMinusTop8, k16, kNumConst };
static __constant__ uint32_t kc[kNumConst] = {1u, 0xffffffffu, 4u, 8u, 32u, 0xffffffe0u,
                                              128u, 0xff000000u, 16u};
__device__ __forceinline__ uint32_t imad(uint32_t a, uint32_t b, uint32_t c) { return a * b + c; }

// Shared-memory accesses by 32-bit shared address.  The rings are accessed
// only through these volatile forms (and cp.async), so their order is kept.
__device__ __forceinline__ uint32_t lds(uint32_t a)
{
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ uint32_t lds_u8(uint32_t a)
{
    uint32_t v;
    asm volatile("ld.shared.u8 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ void sts(uint32_t a, uint32_t v)
{
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(a), "r"(v));
}
// predicated forms: the access happens only when `k` is nonzero (no branch)
__device__ __forceinline__ void lds_if(uint32_t k, uint32_t a, uint32_t &v)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %2, 0;\n\t@p ld.shared.u32 %0, [%1];\n\t}"
                 : "+r"(v)
                 : "r"(a), "r"(k));
}
__device__ __forceinline__ void sts_if(uint32_t k, uint32_t a, uint32_t v)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %2, 0;\n\t@p st.shared.u32 [%0], %1;\n\t}"
                 ::"r"(a), "r"(v), "r"(k));
}
// predicated global stores (no branch): the store happens only when k != 0
__device__ __forceinline__ void stg_if(uint32_t k, uint32_t *p, uint32_t v)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %2, 0;\n\t@p st.global.u32 [%0], %1;\n\t}"
                 ::"l"(p), "r"(v), "r"(k)
                 : "memory");
}
__device__ __forceinline__ void stg64_if(uint32_t k, uint64_t *p, uint64_t v)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %2, 0;\n\t@p st.global.u64 [%0], %1;\n\t}"
                 ::"l"(p), "l"((unsigned long long)v), "r"(k)
                 : "memory");
}

// ---- stream header checks --------------------------------------------------
__host__ __device__ __forceinline__ bool chunk_symbols_valid(uint32_t cs)
{
    return cs >= HUFF_MIN_CHUNK_SYMBOLS && cs <= HUFF_MAX_CHUNK_SYMBOLS && (cs % 16u) == 0;
}

__host__ __device__ __forceinline__ uint64_t ceil_div_u64(uint64_t a, uint64_t b)
{
    return a / b + (a % b != 0);
}

// Launch helpers defined in api.cu.  Devices are numbered below
// kMaxDevices; a call made with a higher ordinal current fails with
// cudaErrorInvalidDevice.
constexpr int kMaxDevices = 64;
int current_device();  // -1 if unreadable or not below kMaxDevices
int device_sm_count();  // SMs of the current device, 0 on error

// One kernel's launch set-up, done once per device under a mutex (several
// host threads may launch at once): the dynamic shared-memory limit when the
// kernel needs more than the 48 KiB default, then the resident CTAs per SM.
struct KernelSetup {
    std::mutex mu;
    std::atomic<int> per_sm[kMaxDevices];
};
cudaError_t kernel_setup(KernelSetup &ks, const void *func, int block, size_t dyn_smem,
                         int *per_sm);

}  // namespace huff

// Kernel launchers (one per translation unit); each returns a cudaError_t.
namespace huff {

// Encoder unit: the granularity of precomputed bit offsets (and of the
// optional per-unit histograms).  16 KiB; u16 counts cannot overflow.
constexpr uint32_t kUnitSymbols = 16384;

cudaError_t launch_histogram(const uint8_t *d_in, uint64_t n, unsigned long long *d_hist,
                             uint16_t *d_unit_hist, cudaStream_t s);
// limit 0: plain Huffman (codes over 32 bits are an error); 1..32: codes of
// at most `limit` bits (package-merge where the Huffman code exceeds it)
cudaError_t launch_build_codebook(const unsigned long long *d_hist, huff_codebook_t *d_cb,
                                  int32_t *d_status, cudaStream_t s, uint32_t limit = 0);
// d_tile_sum: unit_scan_tiles(units) u64 of scratch
cudaError_t launch_unit_offsets(const uint8_t *d_in, uint64_t n, const uint16_t *d_unit_hist,
                                const huff_codebook_t *d_cb, uint32_t *d_unit_bits,
                                unsigned long long *d_unit_off, unsigned long long *d_tile_sum,
                                int32_t *d_status, cudaStream_t s);
// tiles of the unit offset scan (2048 units each)
__host__ __device__ constexpr uint64_t unit_scan_tiles(uint64_t units) { return (units + 2047) / 2048; }
cudaError_t launch_encode(const uint8_t *d_in, uint64_t n, const huff_codebook_t *d_cb,
                          uint32_t cs, uint8_t *d_out, uint64_t out_cap,
                          unsigned long long *d_out_bytes, void *d_ws,
                          const uint16_t *d_unit_hist, int32_t *d_status, cudaStream_t s);
cudaError_t launch_decode(const uint8_t *d_stream, uint64_t bytes, uint8_t *d_out,
                          uint64_t out_cap, unsigned long long *d_n, int32_t *d_status,
                          cudaStream_t s);
uint64_t encode_workspace_bytes(uint64_t n);
}  // namespace huff
