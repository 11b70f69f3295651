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
#include "hist_impl.cuh"

namespace huff {
namespace {

using namespace hst;

constexpr int kHistBlock = kThreads;

__global__ void __launch_bounds__(kHistBlock)
    k_histogram(const uint8_t *__restrict__ in, uint64_t n, unsigned long long *__restrict__ hist,
                uint16_t *__restrict__ unit_hist)
{
    __shared__ __align__(16) uint32_t cnt[256 * 32];
    const int tid = threadIdx.x, lane = tid & 31;
    for (int i = tid; i < 256 * 32; i += kHistBlock)
        cnt[i] = 0;
    const uint32_t col = smem_u32(cnt) + 4u * lane;  // this lane's column
    const uint64_t units = (n + kUnitSymbols - 1) / kUnitSymbols;
    uint32_t prev = 0;  // fold of this thread's bin at the previous unit end
    uint4 a[kVecPerThread];
    uint64_t u = blockIdx.x;
    load_unit(in, n, u, a);
    __syncthreads();
    for (; u < units; u += gridDim.x) {
        uint4 cur[kVecPerThread];
#pragma unroll
        for (int j = 0; j < kVecPerThread; ++j)
            cur[j] = a[j];
        load_unit(in, n, u + gridDim.x, a);  // in flight while this unit is counted
        count_unit(in, n, u, cur, col);
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
    static KernelSetup setup;
    int per_sm = 0;
    err = kernel_setup(setup, (const void *)k_histogram, kHistBlock, 0, &per_sm);
    if (err != cudaSuccess)
        return err;
    const int sms = device_sm_count();
    if (sms < 1)
        return cudaErrorInvalidDevice;
    const uint64_t units = (n + kUnitSymbols - 1) / kUnitSymbols;
    const uint64_t cap = (uint64_t)sms * per_sm;
    const uint64_t grid = units < cap ? units : cap;
    k_histogram<<<(unsigned)grid, kHistBlock, 0, s>>>(d_in, n, d_hist, d_unit_hist);
    return cudaGetLastError();
}

}  // namespace huff
