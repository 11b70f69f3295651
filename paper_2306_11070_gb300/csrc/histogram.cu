// Byte histogram: the "probability of occurrence" step of the paper's
// Huffman Method 1 (Section III-A).
//
// HBM-bound: n bytes read once.  Each CTA keeps 32 private copies of the 256
// counters in shared memory, laid out [bin][lane], and lane l only touches
// column l, so the 32 shared-memory atomics of one warp instruction always
// fall in 32 different banks, whatever the data (a single repeated byte
// included).  Loads are 16-byte, streaming (no L1 allocation), four in flight
// per thread.  At the end every CTA folds its 32 columns and adds one u64 per
// non-zero bin to the global histogram.
#include "huff_internal.cuh"

namespace huff {
namespace {

constexpr int kHistBlock = 512;
constexpr int kHistUnroll = 4;

__device__ __forceinline__ void count_word(uint32_t *col, uint32_t w)
{
    atomicAdd(col + ((w & 0xffu) << 5), 1u);
    atomicAdd(col + (((w >> 8) & 0xffu) << 5), 1u);
    atomicAdd(col + (((w >> 16) & 0xffu) << 5), 1u);
    atomicAdd(col + ((w >> 24) << 5), 1u);
}

__device__ __forceinline__ void count16(uint32_t *col, uint4 v)
{
    count_word(col, v.x);
    count_word(col, v.y);
    count_word(col, v.z);
    count_word(col, v.w);
}

__global__ void __launch_bounds__(kHistBlock)
    k_histogram(const uint8_t *__restrict__ in, uint64_t n, unsigned long long *__restrict__ hist)
{
    __shared__ uint32_t cnt[256 * 32];
    const int lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < 256 * 32; i += kHistBlock)
        cnt[i] = 0;
    __syncthreads();

    uint32_t *col = cnt + lane;
    const uint64_t nvec = n >> 4;
    const uint64_t stride = (uint64_t)gridDim.x * kHistBlock;
    uint64_t i = (uint64_t)blockIdx.x * kHistBlock + threadIdx.x;
    const uint4 *v = reinterpret_cast<const uint4 *>(in);
    for (; i + (kHistUnroll - 1) * stride < nvec; i += kHistUnroll * stride) {
        uint4 a[kHistUnroll];
#pragma unroll
        for (int u = 0; u < kHistUnroll; ++u)
            a[u] = ld_stream16(v + i + u * stride);
#pragma unroll
        for (int u = 0; u < kHistUnroll; ++u)
            count16(col, a[u]);
    }
    for (; i < nvec; i += stride)
        count16(col, ld_stream16(v + i));
    // ragged tail (< 16 bytes)
    const uint64_t g = (uint64_t)blockIdx.x * kHistBlock + threadIdx.x;
    if (g < (n & 15u))
        atomicAdd(col + ((uint32_t)in[(nvec << 4) + g] << 5), 1u);
    __syncthreads();

    // fold the 32 columns of each bin; the rotation keeps the reads of one
    // warp in 32 different banks
    for (int b = threadIdx.x; b < 256; b += kHistBlock) {
        uint32_t s = 0;
#pragma unroll 8
        for (int l = 0; l < 32; ++l)
            s += cnt[(b << 5) + ((l + b) & 31)];
        if (s)
            atomicAdd(hist + b, (unsigned long long)s);
    }
}

}  // namespace

cudaError_t launch_histogram(const uint8_t *d_in, uint64_t n, unsigned long long *d_hist,
                             cudaStream_t s)
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
    const uint64_t nvec = n >> 4;
    uint64_t want = (nvec + (uint64_t)kHistBlock * kHistUnroll - 1) / ((uint64_t)kHistBlock * kHistUnroll);
    uint64_t cap = (uint64_t)device_sm_count() * per_sm;
    uint64_t grid = want < cap ? want : cap;
    if (grid < 1)
        grid = 1;
    k_histogram<<<(unsigned)grid, kHistBlock, 0, s>>>(d_in, n, d_hist);
    return cudaGetLastError();
}

}  // namespace huff
