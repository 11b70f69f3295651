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
//  - k_scan_units: one CTA turns the counts into exclusive prefixes
//    (u64 per unit, plus the total at index `units`).
#include "huff_internal.cuh"

namespace huff {
namespace {

constexpr int kDotBlock = 256;
constexpr int kCountBlock = 256;
constexpr int kScanBlock = 512;
constexpr int kScanPer = 32;  // counts per thread and tile

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

// One CTA scans the unit counts in tiles of kScanBlock * kScanPer units:
// each thread loads its kScanPer consecutive counts with 16-byte loads that
// are all in flight at once, so a tile costs one memory round trip (1 GiB of
// input is 4 tiles), then a block scan of the thread totals and a carry
// across tiles.
__global__ void __launch_bounds__(kScanBlock)
    k_scan_units(const uint32_t *__restrict__ unit_bits, uint64_t units,
                 unsigned long long *__restrict__ unit_off, const int32_t *status)
{
    __shared__ unsigned long long s_warp[kScanBlock / 32];
    __shared__ unsigned long long s_total;
    if (chain_failed(status))
        return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned long long carry = 0;
    for (uint64_t t0 = 0; t0 < units; t0 += (uint64_t)kScanBlock * kScanPer) {
        const uint64_t i = t0 + (uint64_t)kScanPer * tid;
        uint32_t v[kScanPer];
        if (i + kScanPer <= units) {  // i is a multiple of 32: 16-byte aligned
            const uint4 *q = reinterpret_cast<const uint4 *>(unit_bits + i);
#pragma unroll
            for (int j = 0; j < kScanPer / 4; ++j) {
                const uint4 x = q[j];
                v[4 * j] = x.x;
                v[4 * j + 1] = x.y;
                v[4 * j + 2] = x.z;
                v[4 * j + 3] = x.w;
            }
        } else {
#pragma unroll
            for (int j = 0; j < kScanPer; ++j)
                v[j] = i + j < units ? unit_bits[i + j] : 0u;
        }
        unsigned long long own = 0;
#pragma unroll
        for (int j = 0; j < kScanPer; ++j)
            own += v[j];
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
        if (warp == 0) {
            const unsigned long long w = lane < kScanBlock / 32 ? s_warp[lane] : 0ull;
            unsigned long long z = w;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, z, d);
                if (lane >= d)
                    z += y;
            }
            if (lane < kScanBlock / 32)
                s_warp[lane] = z - w;
            if (lane == 31)
                s_total = z;  // the tile total
        }
        __syncthreads();
        unsigned long long run = carry + s_warp[warp] + x - own;
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
        carry += s_total;
        __syncthreads();
    }
    if (tid == 0)
        unit_off[units] = carry;
}

}  // namespace

cudaError_t launch_unit_offsets(const uint8_t *d_in, uint64_t n, const uint16_t *d_unit_hist,
                                const huff_codebook_t *d_cb, uint32_t *d_unit_bits,
                                unsigned long long *d_unit_off, int32_t *d_status, cudaStream_t s)
{
    const uint64_t units = (n + kUnitSymbols - 1) / kUnitSymbols;
    if (units == 0)
        return cudaMemsetAsync(d_unit_off, 0, sizeof(unsigned long long), s);
    const int sms = device_sm_count();
    if (d_unit_hist) {
        uint64_t grid = (units + (kDotBlock / 32) - 1) / (kDotBlock / 32);
        if (grid > (uint64_t)sms * 8)
            grid = (uint64_t)sms * 8;
        k_unit_bits_hist<<<(unsigned)grid, kDotBlock, 0, s>>>(d_unit_hist, units, d_cb, d_unit_bits,
                                                              d_status);
    } else {
        static int per_sm = 0;
        if (per_sm == 0) {
            cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_unit_bits_input,
                                                                            kCountBlock, 0);
            if (err != cudaSuccess)
                return err;
            if (per_sm < 1)
                per_sm = 1;
        }
        uint64_t grid = units < (uint64_t)sms * per_sm ? units : (uint64_t)sms * per_sm;
        k_unit_bits_input<<<(unsigned)grid, kCountBlock, 0, s>>>(d_in, n, d_cb, d_unit_bits,
                                                                 d_status);
    }
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess)
        return err;
    k_scan_units<<<1, kScanBlock, 0, s>>>(d_unit_bits, units, d_unit_off, d_status);
    return cudaGetLastError();
}

}  // namespace huff
