// Device-wide scan and stable LSD radix passes, the building blocks of the
// block-sorting transform (Method 3).
//
//  - scan: exclusive or inclusive prefix sum of u32 in three launches (tile
//    sums; one CTA scans the tile sums and writes the total; every tile adds
//    its offset), tiles of 4096 elements.
//  - radix pass: stable scatter of (u64 key, u32 value) pairs by the 8-bit
//    digit (key >> shift) & 255, in three launches: per-tile digit counts
//    stored digit-major (count[d * tiles + t]), their exclusive scan (which
//    is then each tile's first output slot per digit, tiles in order within
//    a digit: stability across tiles), and the scatter.  The scatter ranks
//    equal digits inside a tile in element order with __match_any_sync per
//    warp step and per-warp running counts, sorts the tile in shared memory
//    and writes it out digit run by digit run, so consecutive threads write
//    consecutive slots.
// All loops are bounded by the element count; nothing waits on another CTA.
#pragma once

#include "huff_internal.cuh"

namespace huff {
namespace srt {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr uint32_t kScanTile = kScanThreads * kScanItems;  // 4096
constexpr int kRadixThreads = 256;
constexpr int kRadixItems = 8;
constexpr uint32_t kRadixTile = kRadixThreads * kRadixItems;  // 2048
constexpr int kRadixWarps = kRadixThreads / 32;

__host__ __device__ inline uint32_t div_up(uint64_t a, uint32_t b) { return (uint32_t)((a + b - 1) / b); }

// ---- scan -----------------------------------------------------------------
// block-wide exclusive scan of one value per thread (kScanThreads threads);
// returns the exclusive prefix, *total gets the sum
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *warp_sums, uint32_t &total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d)
            x += y;
    }
    if (lane == 31)
        warp_sums[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t s = lane < kScanThreads / 32 ? warp_sums[lane] : 0u;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, s, d);
            if (lane >= d)
                s += y;
        }
        if (lane < kScanThreads / 32)
            warp_sums[lane] = s;  // inclusive warp prefix
    }
    __syncthreads();
    total = warp_sums[kScanThreads / 32 - 1];
    const uint32_t before = w > 0 ? warp_sums[w - 1] : 0u;
    __syncthreads();  // warp_sums reusable after return
    return before + x - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const uint32_t *in, uint32_t count,
                                                             uint32_t *part)
{
    __shared__ uint32_t ws[kScanThreads / 32];
    const uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j)
        if (base + j < count)
            s += in[base + j];
    uint32_t total;
    block_excl_scan(s, ws, total);
    if (threadIdx.x == 0)
        part[blockIdx.x] = total;
}

// one CTA: exclusive scan of the tile sums in place, the total to *total
__global__ void __launch_bounds__(kScanThreads) k_scan_parts(uint32_t *part, uint32_t tiles,
                                                             uint32_t *total)
{
    __shared__ uint32_t ws[kScanThreads / 32];
    uint32_t carry = 0;
    for (uint32_t b = 0; b < tiles; b += kScanThreads) {
        const uint32_t i = b + threadIdx.x;
        const uint32_t v = i < tiles ? part[i] : 0u;
        uint32_t t;
        const uint32_t x = block_excl_scan(v, ws, t);
        if (i < tiles)
            part[i] = carry + x;
        carry += t;
    }
    if (threadIdx.x == 0 && total)
        *total = carry;
}

template <bool kInclusive>
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const uint32_t *in, uint32_t count,
                                                             const uint32_t *part, uint32_t *out)
{
    __shared__ uint32_t ws[kScanThreads / 32];
    const uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        v[j] = base + j < count ? in[base + j] : 0u;
        s += v[j];
    }
    uint32_t total;
    uint32_t run = part[blockIdx.x] + block_excl_scan(s, ws, total);
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        if (base + j < count)
            out[base + j] = kInclusive ? run + v[j] : run;
        run += v[j];
    }
}

inline uint64_t scan_parts_bytes(uint64_t count) { return 4ull * div_up(count, kScanTile) + 16; }

// out[i] = sum of in[0, i) (or [0, i]); *d_total = sum of all (if given).
// `part` holds scan_parts_bytes(count).  in == out is allowed.
inline cudaError_t scan_u32(const uint32_t *in, uint32_t *out, uint32_t count, bool inclusive,
                            uint32_t *part, uint32_t *d_total, cudaStream_t s)
{
    const uint32_t tiles = div_up(count, kScanTile);
    if (tiles > 0) {
        k_scan_tiles<<<tiles, kScanThreads, 0, s>>>(in, count, part);
    }
    k_scan_parts<<<1, kScanThreads, 0, s>>>(part, tiles, d_total);
    if (tiles > 0) {
        if (inclusive)
            k_scan_apply<true><<<tiles, kScanThreads, 0, s>>>(in, count, part, out);
        else
            k_scan_apply<false><<<tiles, kScanThreads, 0, s>>>(in, count, part, out);
    }
    return cudaGetLastError();
}

// ---- radix pass -----------------------------------------------------------
__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}
__device__ __forceinline__ uint32_t lanemask_le()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_le;" : "=r"(m));
    return m;
}

__global__ void __launch_bounds__(kRadixThreads) k_radix_count(const uint64_t *keys, uint32_t count,
                                                               uint32_t shift, uint32_t *hist,
                                                               uint32_t tiles)
{
    __shared__ uint32_t c[256];
    c[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t base = (uint64_t)blockIdx.x * kRadixTile;
    const int lane = threadIdx.x & 31;
    uint32_t dig[kRadixItems];
#pragma unroll
    for (int j = 0; j < kRadixItems; ++j) {  // every load in flight before the first use
        const uint64_t e = base + (uint64_t)j * kRadixThreads + threadIdx.x;
        dig[j] = e < count ? (uint32_t)(keys[e] >> shift) & 255u : 256u;
    }
#pragma unroll
    for (int j = 0; j < kRadixItems; ++j) {
        const uint32_t d = dig[j];
        const bool ok = d < 256u;
        const uint32_t mask = __match_any_sync(0xffffffffu, d);
        // one shared add per distinct digit of the warp step
        if (ok && lane == __ffs(mask) - 1)
            atomicAdd(&c[d], (uint32_t)__popc(mask));
    }
    __syncthreads();
    hist[(uint64_t)threadIdx.x * tiles + blockIdx.x] = c[threadIdx.x];
}

__global__ void __launch_bounds__(kRadixThreads) k_radix_scatter(
    const uint64_t *kin, const uint32_t *vin, uint64_t *kout, uint32_t *vout, uint32_t count,
    uint32_t shift, const uint32_t *offs, uint32_t tiles)
{
    __shared__ uint64_t sk[kRadixTile];
    __shared__ uint32_t sv[kRadixTile];
    __shared__ uint32_t wcnt[kRadixWarps][256];
    __shared__ uint32_t dstart[256];
    __shared__ uint32_t gbase[256];
    __shared__ uint32_t ws[kRadixWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kRadixWarps * 256; i += kRadixThreads)
        (&wcnt[0][0])[i] = 0;
    __syncthreads();
    // warp w owns the tile's elements [w * 256, (w + 1) * 256), taken 32 at
    // a time in order, so ranks follow element order
    const uint64_t base = (uint64_t)blockIdx.x * kRadixTile + (uint64_t)w * (kRadixItems * 32);
    uint64_t key[kRadixItems];
    uint32_t val[kRadixItems], rank[kRadixItems];
#pragma unroll
    for (int j = 0; j < kRadixItems; ++j) {  // every load in flight before the first use
        const uint64_t e = base + (uint64_t)j * 32 + lane;
        const bool ok = e < count;
        key[j] = ok ? kin[e] : 0ull;
        val[j] = ok ? vin[e] : 0u;
    }
#pragma unroll
    for (int j = 0; j < kRadixItems; ++j) {
        const uint64_t e = base + (uint64_t)j * 32 + lane;
        const bool ok = e < count;
        const uint32_t d = ok ? (uint32_t)(key[j] >> shift) & 255u : 256u;
        const uint32_t mask = __match_any_sync(0xffffffffu, d);
        rank[j] = ok ? wcnt[w][d & 255u] + __popc(mask & lanemask_lt()) : 0u;
        __syncwarp();
        if (ok && lane == __ffs(mask) - 1)
            wcnt[w][d] += __popc(mask);
        __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive prefix over the warps, then over the digits
    {
        const uint32_t d = threadIdx.x;  // kRadixThreads == 256 digits
        uint32_t run = 0;
#pragma unroll
        for (int ww = 0; ww < kRadixWarps; ++ww) {
            const uint32_t t = wcnt[ww][d];
            wcnt[ww][d] = run;
            run += t;
        }
        // block scan of the 256 digit totals (8 warps)
        uint32_t x = run;
#pragma unroll
        for (int s = 1; s < 32; s <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, s);
            if (lane >= s)
                x += y;
        }
        if (lane == 31)
            ws[w] = x;
        __syncthreads();
        uint32_t before = 0;
        for (int ww = 0; ww < w; ++ww)
            before += ws[ww];
        dstart[d] = before + x - run;
        gbase[d] = offs[(uint64_t)d * tiles + blockIdx.x];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kRadixItems; ++j) {
        const uint64_t e = base + (uint64_t)j * 32 + lane;
        if (e < count) {
            const uint32_t d = (uint32_t)(key[j] >> shift) & 255u;
            const uint32_t q = dstart[d] + wcnt[w][d] + rank[j];
            sk[q] = key[j];
            sv[q] = val[j];
        }
    }
    __syncthreads();
    const uint64_t tb = (uint64_t)blockIdx.x * kRadixTile;
    const uint32_t n_here = (uint32_t)(count - tb < kRadixTile ? count - tb : kRadixTile);
    for (uint32_t q = threadIdx.x; q < n_here; q += kRadixThreads) {
        const uint64_t k = sk[q];
        const uint32_t d = (uint32_t)(k >> shift) & 255u;
        const uint64_t dst = (uint64_t)gbase[d] + (q - dstart[d]);
        kout[dst] = k;
        vout[dst] = sv[q];
    }
}

// scratch of one radix pass: the digit counts (scanned in place) and the
// scan's tile sums
inline uint64_t radix_scratch_bytes(uint64_t count)
{
    const uint64_t hist = 256ull * div_up(count, kRadixTile);
    return ((4 * hist + 255) & ~255ull) + scan_parts_bytes(hist);
}

// Stable sort of (k, v)[0, count) by the key bits [lo, hi) in passes of 8
// bits, ping-ponging between (k0, v0) and (k1, v1).  Returns in `flip`
// whether the result ended in (k1, v1).
inline cudaError_t radix_sort_bits(uint64_t *k0, uint32_t *v0, uint64_t *k1, uint32_t *v1,
                                   uint32_t count, uint32_t lo, uint32_t hi, void *scratch,
                                   cudaStream_t s, bool &flip)
{
    flip = false;
    if (count <= 1)
        return cudaSuccess;
    const uint32_t tiles = div_up(count, kRadixTile);
    uint32_t *hist = static_cast<uint32_t *>(scratch);
    const uint64_t hist_n = 256ull * tiles;
    uint32_t *part = reinterpret_cast<uint32_t *>(static_cast<uint8_t *>(scratch) +
                                                  ((4 * hist_n + 255) & ~255ull));
    for (uint32_t sh = lo; sh < hi; sh += 8) {
        uint64_t *ki = flip ? k1 : k0;
        uint32_t *vi = flip ? v1 : v0;
        uint64_t *ko = flip ? k0 : k1;
        uint32_t *vo = flip ? v0 : v1;
        k_radix_count<<<tiles, kRadixThreads, 0, s>>>(ki, count, sh, hist, tiles);
        cudaError_t e = scan_u32(hist, hist, (uint32_t)hist_n, false, part, nullptr, s);
        if (e != cudaSuccess)
            return e;
        k_radix_scatter<<<tiles, kRadixThreads, 0, s>>>(ki, vi, ko, vo, count, sh, hist, tiles);
        flip = !flip;
    }
    return cudaGetLastError();
}

}  // namespace srt
}  // namespace huff
