// Byte histogram: the "probability of occurrence" step of the paper's
// Huffman Method 1 (Section III-A).
//
// HBM-bound: n bytes read once.  Each CTA keeps 32 private copies of the 256
// counters in shared memory, laid out [bin][lane], and lane l only touches
// column l, so the 32 shared-memory atomics of one warp instruction always
// fall in 32 different banks, whatever the data (a single repeated byte
// included).  Persistent CTAs take 16 KiB units round robin; each thread
// loads its four 16-byte pieces of the next unit before counting the current
// one.
//
// Optionally the kernel also writes every unit's own histogram (u16[256],
// 512 bytes per 16 KiB): the encoder turns these into the bit offset of each
// unit with a dot product against the code lengths, so it never has to wait
// on another CTA.  A unit's counts are the difference of two folds of the
// running columns, so the columns are never cleared.
#include "huff_internal.cuh"

namespace huff {
namespace {

constexpr int kHistBlock = 256;
constexpr int kVecPerThread = kUnitSymbols / 16 / kHistBlock;  // 4

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

// Sum of bin `tid` over its 32 columns; the rotation keeps one warp's reads
// in distinct banks.
__device__ __forceinline__ uint32_t fold_bin(const uint32_t *cnt, int tid)
{
    uint32_t s = 0;
#pragma unroll
    for (int l = 0; l < 32; ++l)
        s += cnt[(tid << 5) + ((l + tid) & 31)];
    return s;
}

__global__ void __launch_bounds__(kHistBlock)
    k_histogram(const uint8_t *__restrict__ in, uint64_t n, unsigned long long *__restrict__ hist,
                uint16_t *__restrict__ unit_hist)
{
    __shared__ uint32_t cnt[256 * 32];
    const int tid = threadIdx.x, lane = tid & 31;
    for (int i = tid; i < 256 * 32; i += kHistBlock)
        cnt[i] = 0;
    const uint32_t col = smem_u32(cnt) + 4u * lane;  // this lane's column
    const uint64_t units = (n + kUnitSymbols - 1) / kUnitSymbols;
    const uint64_t nvec = n >> 4;
    const uint4 *v = reinterpret_cast<const uint4 *>(in);
    uint32_t prev = 0;  // fold of this thread's bin at the previous unit end
    uint4 a[kVecPerThread];
    auto load_unit = [&](uint64_t uu) {
#pragma unroll
        for (int j = 0; j < kVecPerThread; ++j) {
            const uint64_t q = uu * (kUnitSymbols / 16) + j * kHistBlock + tid;
            a[j] = (uu < units && q < nvec) ? ld_stream16(v + q) : make_uint4(0, 0, 0, 0);
        }
    };
    uint64_t u = blockIdx.x;
    load_unit(u);
    __syncthreads();
    for (; u < units; u += gridDim.x) {
        uint4 cur[kVecPerThread];
#pragma unroll
        for (int j = 0; j < kVecPerThread; ++j)
            cur[j] = a[j];
        load_unit(u + gridDim.x);  // in flight while this unit is counted
#pragma unroll
        for (int j = 0; j < kVecPerThread; ++j) {
            const uint64_t q = u * (kUnitSymbols / 16) + j * kHistBlock + tid;
            if (q < nvec)
                count16(col, cur[j]);
        }
        if (u == units - 1) {  // ragged tail (< 16 bytes) belongs to the last unit
            if (tid < (int)(n & 15u))
                count_at(col, in[(nvec << 4) + tid]);
        }
        if (unit_hist) {
            __syncthreads();  // all counts of unit u are in
            const uint32_t s = fold_bin(cnt, tid);
            unit_hist[u * 256 + tid] = (uint16_t)(s - prev);
            prev = s;
            __syncthreads();  // folds read before the next unit's counts
        }
    }
    __syncthreads();
    const uint32_t s = fold_bin(cnt, tid);
    if (s)
        atomicAdd(hist + tid, (unsigned long long)s);
}

}  // namespace

cudaError_t launch_histogram(const uint8_t *d_in, uint64_t n, unsigned long long *d_hist,
                             uint16_t *d_unit_hist, cudaStream_t s)
{
    cudaError_t err = cudaMemsetAsync(d_hist, 0, 256 * sizeof(unsigned long long), s);
    if (err != cudaSuccess || n == 0)
        return err;
    static int per_sm = 0;
    if (per_sm == 0) {
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_histogram, kHistBlock, 0);
        if (err != cudaSuccess)
            return err;
        if (per_sm < 1)
            per_sm = 1;
    }
    const uint64_t units = (n + kUnitSymbols - 1) / kUnitSymbols;
    const uint64_t cap = (uint64_t)device_sm_count() * per_sm;
    const uint64_t grid = units < cap ? units : cap;
    k_histogram<<<(unsigned)grid, kHistBlock, 0, s>>>(d_in, n, d_hist, d_unit_hist);
    return cudaGetLastError();
}

}  // namespace huff
