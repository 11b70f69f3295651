// Histogram device routines (CTAs of 256 threads, 16 KiB units), shared by
// the single-stream kernel (histogram.cu) and the batched kernel (batch.cu).
// See histogram.cu for the method.
#pragma once

#include "huff_internal.cuh"

namespace huff {
namespace hst {

constexpr int kThreads = 256;
constexpr int kVecPerThread = kUnitSymbols / 16 / kThreads;  // 4

// One count: a shared-memory reduction at the 32-bit shared address of
// (byte, lane); byte * 128 is the row offset of the [byte][lane] layout.
__device__ __forceinline__ void count_at(uint32_t col, uint32_t byte)
{
    asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(col + (byte << 7)) : "memory");
}

__device__ __forceinline__ void count_word(uint32_t col, uint32_t w)
{
    count_at(col, __byte_perm(w, 0u, 0x4440u));
    count_at(col, __byte_perm(w, 0u, 0x4441u));
    count_at(col, __byte_perm(w, 0u, 0x4442u));
    count_at(col, __byte_perm(w, 0u, 0x4443u));
}

__device__ __forceinline__ void count16(uint32_t col, uint4 v)
{
    count_word(col, v.x);
    count_word(col, v.y);
    count_word(col, v.z);
    count_word(col, v.w);
}

// Sum of bin `tid` over its 32 columns, in eight 16-byte loads.  The
// rotation spreads one warp's loads over all eight 16-byte bank groups (four
// lanes per group, the minimum for 512 bytes).
__device__ __forceinline__ uint32_t fold_bin(const uint32_t *cnt, int tid)
{
    const uint4 *row = reinterpret_cast<const uint4 *>(cnt + (tid << 5));
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const uint4 v = row[(j + tid) & 7];
        s += (v.x + v.y) + (v.z + v.w);
    }
    return s;
}

// The calling thread's four 16-byte pieces of unit u of (in, n).
__device__ __forceinline__ void load_unit(const uint8_t *in, uint64_t n, uint64_t u,
                                          uint4 (&a)[kVecPerThread])
{
    const uint64_t units = (n + kUnitSymbols - 1) / kUnitSymbols;
    const uint64_t nvec = n >> 4;
    const uint4 *v = reinterpret_cast<const uint4 *>(in);
#pragma unroll
    for (int j = 0; j < kVecPerThread; ++j) {
        const uint64_t q = u * (kUnitSymbols / 16) + j * kThreads + threadIdx.x;
        a[j] = (u < units && q < nvec) ? ld_stream16(v + q) : make_uint4(0, 0, 0, 0);
    }
}

// Count the loaded pieces of unit u (and, for the last unit, the < 16-byte
// tail) into the lane's column.
__device__ __forceinline__ void count_unit(const uint8_t *in, uint64_t n, uint64_t u,
                                           const uint4 (&a)[kVecPerThread], uint32_t col)
{
    const uint64_t units = (n + kUnitSymbols - 1) / kUnitSymbols;
    const uint64_t nvec = n >> 4;
#pragma unroll
    for (int j = 0; j < kVecPerThread; ++j) {
        const uint64_t q = u * (kUnitSymbols / 16) + j * kThreads + threadIdx.x;
        if (q < nvec)
            count16(col, a[j]);
    }
    if (u == units - 1 && threadIdx.x < (n & 15u))
        count_at(col, in[(nvec << 4) + threadIdx.x]);
}

}  // namespace hst
}  // namespace huff
