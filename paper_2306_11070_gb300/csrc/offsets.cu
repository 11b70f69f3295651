// Bit offsets of the encoder's 16 KiB units.
//
// The paper's Method 2 (Section III-A) codes segments independently and
// reassembles them by id; here all units share one codebook and one
// bitstream, so unit u starts at the total code length of units 0..u-1.
// These kernels compute that prefix before the encoder runs, which lets
// every encoder CTA write its unit with no cross-CTA wait:
//  - k_unit_bits_hist: a unit's bit count is the dot product of its byte
//    histogram (from the histogram pass) with the code lengths -- a warp per
//    unit, 512 bytes read per 16 KiB unit;
//  - k_unit_bits_input: without those histograms, the same count straight
//    from the input (one HBM read of the input, per-lane replicated length
//    table in shared memory);
//  - k_scan_tile_sums + k_scan_apply: the counts become exclusive
//    prefixes (u64 per unit, plus the total at index `units`).
#include "huff_internal.cuh"

namespace huff {
namespace {

constexpr int kDotBlock = 256;
constexpr int kCountBlock = 256;

__global__ void __launch_bounds__(kDotBlock)
    k_unit_bits_hist(const uint16_t *__restrict__ unit_hist, uint64_t units,
                     const huff_codebook_t *__restrict__ cb, uint32_t *__restrict__ unit_bits,
                     const int32_t *status)
{
    __shared__ uint32_t len[256];
    if (chain_failed(status))
        return;
    len[threadIdx.x] = cb->len[threadIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint64_t nwarps = (uint64_t)gridDim.x * (kDotBlock / 32);
    for (uint64_t u = ((uint64_t)blockIdx.x * kDotBlock + threadIdx.x) >> 5; u < units; u += nwarps) {
        const uint4 q = reinterpret_cast<const uint4 *>(unit_hist + u * 256)[lane];
        const uint32_t w[4] = {q.x, q.y, q.z, q.w};
        uint32_t s = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            s += (w[j] & 0xffffu) * len[lane * 8 + 2 * j] + (w[j] >> 16) * len[lane * 8 + 2 * j + 1];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1)
            s += __shfl_xor_sync(0xffffffffu, s, d);
        if (lane == 0)
            unit_bits[u] = s;
    }
}

__global__ void __launch_bounds__(kCountBlock)
    k_unit_bits_input(const uint8_t *__restrict__ in, uint64_t n,
                      const huff_codebook_t *__restrict__ cb, uint32_t *__restrict__ unit_bits,
                      const int32_t *status)
{
    __shared__ uint32_t len[256 * 32];  // [byte][lane]
    __shared__ uint32_t s_warp[kCountBlock / 32];
    if (chain_failed(status))
        return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < 256 * 32; i += kCountBlock)
        len[i] = cb->len[i >> 5];
    __syncthreads();
    const uint64_t units = (n + kUnitSymbols - 1) / kUnitSymbols;
    const uint64_t nvec = n >> 4;
    const uint4 *v = reinterpret_cast<const uint4 *>(in);
    constexpr int kVec = kUnitSymbols / 16 / kCountBlock;  // 4
    for (uint64_t u = blockIdx.x; u < units; u += gridDim.x) {
        uint32_t s = 0;
        uint4 a[kVec];
#pragma unroll
        for (int j = 0; j < kVec; ++j) {
            const uint64_t q = u * (kUnitSymbols / 16) + j * kCountBlock + tid;
            a[j] = q < nvec ? ld_stream16(v + q) : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int j = 0; j < kVec; ++j) {
            const uint64_t q = u * (kUnitSymbols / 16) + j * kCountBlock + tid;
            if (q < nvec) {
                const uint32_t w[4] = {a[j].x, a[j].y, a[j].z, a[j].w};
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    s += len[(((w[k >> 2] >> (8 * (k & 3))) & 0xffu) << 5) | lane];
            }
        }
        if (u == units - 1 && tid < (int)(n & 15u))
            s += len[((uint32_t)in[(nvec << 4) + tid] << 5) | lane];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1)
            s += __shfl_xor_sync(0xffffffffu, s, d);
        if (lane == 0)
            s_warp[warp] = s;
        __syncthreads();
        if (tid == 0) {
            uint32_t t = 0;
#pragma unroll
            for (int w = 0; w < kCountBlock / 32; ++w)
                t += s_warp[w];
            unit_bits[u] = t;
        }
        __syncthreads();
    }
}

// The exclusive scan of the unit counts in two launches over tiles of
// kScanTile units (one CTA per tile, each thread kScanPer consecutive counts
// loaded with 16-byte loads that are all in flight at once):
//  - k_scan_tile_sums: every tile's total;
//  - k_scan_apply: every tile adds up the totals of the tiles before it (a
//    few dozen at 1 GiB), scans its own counts and writes the u64 offsets;
//    the last tile also writes the grand total at index `units`.
constexpr int kScanThreads = 256;
constexpr int kScanPer = 8;
constexpr uint32_t kScanTile = kScanThreads * kScanPer;  // 2048 units

__device__ __forceinline__ void load_counts(const uint32_t *unit_bits, uint64_t units, uint64_t i,
                                            uint32_t (&v)[kScanPer])
{
    if (i + kScanPer <= units) {  // i is a multiple of 8: 16-byte aligned
        const uint4 *q = reinterpret_cast<const uint4 *>(unit_bits + i);
        const uint4 x0 = q[0], x1 = q[1];
        v[0] = x0.x, v[1] = x0.y, v[2] = x0.z, v[3] = x0.w;
        v[4] = x1.x, v[5] = x1.y, v[6] = x1.z, v[7] = x1.w;
    } else {
#pragma unroll
        for (int j = 0; j < kScanPer; ++j)
            v[j] = i + j < units ? unit_bits[i + j] : 0u;
    }
}

// block-wide exclusive scan of one u64 per thread; *total the sum
__device__ __forceinline__ unsigned long long block_scan_u64(unsigned long long own,
                                                             unsigned long long *s_warp,
                                                             unsigned long long &total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long x = own;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d)
            x += y;
    }
    if (lane == 31)
        s_warp[warp] = x;
    __syncthreads();
    unsigned long long before = 0, all = 0;
#pragma unroll
    for (int w = 0; w < kScanThreads / 32; ++w) {
        const unsigned long long t = s_warp[w];
        before += w < warp ? t : 0ull;
        all += t;
    }
    total = all;
    return before + x - own;
}

__global__ void __launch_bounds__(kScanThreads)
    k_scan_tile_sums(const uint32_t *__restrict__ unit_bits, uint64_t units,
                     unsigned long long *__restrict__ tile_sum, const int32_t *status)
{
    __shared__ unsigned long long s_warp[kScanThreads / 32];
    if (chain_failed(status))
        return;
    uint32_t v[kScanPer];
    load_counts(unit_bits, units, (uint64_t)blockIdx.x * kScanTile + (uint64_t)kScanPer * threadIdx.x,
                v);
    unsigned long long own = 0;
#pragma unroll
    for (int j = 0; j < kScanPer; ++j)
        own += v[j];
    unsigned long long total;
    block_scan_u64(own, s_warp, total);
    if (threadIdx.x == 0)
        tile_sum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads)
    k_scan_apply(const uint32_t *__restrict__ unit_bits, uint64_t units,
                 const unsigned long long *__restrict__ tile_sum,
                 unsigned long long *__restrict__ unit_off, const int32_t *status)
{
    __shared__ unsigned long long s_warp[kScanThreads / 32];
    __shared__ unsigned long long s_base;
    if (chain_failed(status))
        return;
    // the totals of the tiles before this one
    unsigned long long b = 0;
    for (uint32_t t = threadIdx.x; t < blockIdx.x; t += kScanThreads)
        b += tile_sum[t];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1)
        b += __shfl_xor_sync(0xffffffffu, b, d);
    if (threadIdx.x == 0)
        s_base = 0;
    __syncthreads();
    if ((threadIdx.x & 31) == 0 && b)
        atomicAdd(&s_base, b);
    const uint64_t i = (uint64_t)blockIdx.x * kScanTile + (uint64_t)kScanPer * threadIdx.x;
    uint32_t v[kScanPer];
    load_counts(unit_bits, units, i, v);
    unsigned long long own = 0;
#pragma unroll
    for (int j = 0; j < kScanPer; ++j)
        own += v[j];
    unsigned long long total;
    const unsigned long long x = block_scan_u64(own, s_warp, total);  // has a barrier
    unsigned long long run = s_base + x;
    if (i + kScanPer <= units) {
#pragma unroll
        for (int j = 0; j < kScanPer; j += 2) {
            const unsigned long long a = run;
            run += v[j];
            reinterpret_cast<ulonglong2 *>(unit_off + i)[j / 2] = make_ulonglong2(a, run);
            run += v[j + 1];
        }
    } else {
#pragma unroll
        for (int j = 0; j < kScanPer; ++j) {
            if (i + j < units)
                unit_off[i + j] = run;
            run += v[j];
        }
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0)
        unit_off[units] = s_base + total;
}

}  // namespace

cudaError_t launch_unit_offsets(const uint8_t *d_in, uint64_t n, const uint16_t *d_unit_hist,
                                const huff_codebook_t *d_cb, uint32_t *d_unit_bits,
                                unsigned long long *d_unit_off, unsigned long long *d_tile_sum,
                                int32_t *d_status, cudaStream_t s)
{
    const uint64_t units = (n + kUnitSymbols - 1) / kUnitSymbols;
    if (units == 0)
        return cudaMemsetAsync(d_unit_off, 0, sizeof(unsigned long long), s);
    const int sms = device_sm_count();
    if (sms < 1)
        return cudaErrorInvalidDevice;
    if (d_unit_hist) {
        uint64_t grid = (units + (kDotBlock / 32) - 1) / (kDotBlock / 32);
        if (grid > (uint64_t)sms * 8)
            grid = (uint64_t)sms * 8;
        k_unit_bits_hist<<<(unsigned)grid, kDotBlock, 0, s>>>(d_unit_hist, units, d_cb, d_unit_bits,
                                                              d_status);
    } else {
        static KernelSetup setup;
        int per_sm = 0;
        const cudaError_t err =
            kernel_setup(setup, (const void *)k_unit_bits_input, kCountBlock, 0, &per_sm);
        if (err != cudaSuccess)
            return err;
        uint64_t grid = units < (uint64_t)sms * per_sm ? units : (uint64_t)sms * per_sm;
        k_unit_bits_input<<<(unsigned)grid, kCountBlock, 0, s>>>(d_in, n, d_cb, d_unit_bits,
                                                                 d_status);
    }
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess)
        return err;
    static_assert(kScanTile == 2048, "unit_scan_tiles assumes 2048-unit tiles");
    const uint32_t tiles = (uint32_t)unit_scan_tiles(units);
    k_scan_tile_sums<<<tiles, kScanThreads, 0, s>>>(d_unit_bits, units, d_tile_sum, d_status);
    k_scan_apply<<<tiles, kScanThreads, 0, s>>>(d_unit_bits, units, d_tile_sum, d_unit_off,
                                                d_status);
    return cudaGetLastError();
}

}  // namespace huff
