// Method 3 (Section III-A): the block-sorting (Burrows-Wheeler) transform of
// every block before Method 2's coder, its inverse, and the Method 3
// container.
//
// Forward: the rotations of all blocks are sorted at once by prefix
// doubling.  Every position i carries a rank RK[i] = the first sorted slot
// of its group (the rotations that agree on the prefix compared so far);
// slots of block b are [b * block, b * block + m_b), so ranks are global.
//   round 0: sort all positions by (block, first 4 bytes of the rotation);
//   round r: with h = 4 * 2^(r-1), the still-unresolved positions (groups of
//            more than one) are sorted by (group, RK[i + h within the block])
//            and their groups split where that second rank changes;
// until no group has two members or the compared prefix covers the longest
// block (then the remaining groups are equal rotations, already in start
// order since every pass is stable and the first order is by position).
// The sorts are stable LSD radix passes over only the key bits in use.  In
// rounds r >= 1 the active list is already in group order, so only each
// group's members need sorting: groups that fit one CTA's window (most of
// them on text) are sorted in shared memory in place, and only the members
// of the larger groups go through the global radix passes.
//
// Inverse: LF[p] = the slot of row p's last byte in a stable sort of the
// last column by (block, byte); the block is the walk p -> LF[p] from the
// primary row, emitted backwards.  The walk is cut at sample rows (every
// 64th row and the primary rows): each sample walks to the next sample and
// records the distance, list ranking by pointer jumping over the samples
// gives each sample's distance from the primary row, and every sample then
// re-walks its stretch writing the bytes in place.  A periodic block's walk
// returns to the primary row after one period c; the rest of the block
// repeats it.
#include "api_trace.h"
#include "sort_impl.cuh"

namespace huff {
namespace {

using namespace srt;

constexpr int kEw = 256;               // threads of the elementwise kernels
constexpr uint32_t kSampleGap = 64;    // rows between regular samples
constexpr uint32_t kNil = 0xffffffffu;

unsigned ew_grid(uint64_t count)
{
    const uint64_t cap = (uint64_t)device_sm_count() * 16;
    uint64_t g = (count + kEw - 1) / kEw;
    if (g > cap)
        g = cap;
    return (unsigned)(g < 1 ? 1 : g);
}

uint32_t bit_width(uint64_t v)
{
    uint32_t b = 0;
    while (v) {
        ++b;
        v >>= 1;
    }
    return b;
}

__device__ __forceinline__ void block_span(uint32_t i, uint32_t block, uint32_t n, uint32_t &s,
                                           uint32_t &m)
{
    s = (i / block) * block;
    m = n - s < block ? n - s : block;
}

// ---- forward --------------------------------------------------------------
// round 0 keys: (block id, big-endian first 4 bytes of the rotation)
__global__ void k_bwt_init(const uint8_t *x, uint32_t n, uint32_t block, uint64_t *key,
                           uint32_t *val, uint32_t *act)
{
    for (uint32_t i = blockIdx.x * kEw + threadIdx.x; i < n; i += gridDim.x * kEw) {
        uint32_t s, m;
        block_span(i, block, n, s, m);
        const uint32_t r = i - s;
        uint32_t k = 0;
#pragma unroll
        for (uint32_t t = 0; t < 4; ++t)
            k = (k << 8) | x[s + (uint32_t)(((uint64_t)r + t) % m)];
        key[i] = ((uint64_t)(i / block) << 32) | k;
        val[i] = i;
        act[i] = i;
    }
}

// round r keys: (group, rank of the rotation h bytes on, relative to the
// block), packed so that the passes cover only the bits in use
__global__ void k_bwt_round_keys(const uint32_t *sa, const uint32_t *rk, const uint32_t *act,
                                 const uint32_t *grp, uint32_t count, uint32_t n, uint32_t block,
                                 uint64_t h, uint32_t lo_bits, uint64_t *key, uint32_t *val)
{
    for (uint32_t k = blockIdx.x * kEw + threadIdx.x; k < count; k += gridDim.x * kEw) {
        const uint32_t i = sa[act[k]];
        uint32_t s, m;
        block_span(i, block, n, s, m);
        const uint32_t j = s + (uint32_t)(((uint64_t)(i - s) + h) % m);
        key[k] = ((uint64_t)grp[k] << lo_bits) | (rk[j] - s);
        val[k] = i;
    }
}

// ---- sorting the small groups of a round in shared memory ------------------
// The active list of round r >= 1 is in group order (its keys' high bits, the
// group number, never decrease), so sorting it means sorting every group's
// members by the low bits.  CTA t takes the groups that start in the window
// [t W, (t+1) W) of the list; they end before the first group start of the
// next window, so its range [a, b) is at most 2 W long, unless the last group
// starting in the window runs past the next one: such a group (more than W
// members) is left out (range [a, L)) and marked uncovered for the global
// passes.  Sorting within groups keeps every key's group bits at its index,
// so the start tests of neighbouring CTAs read the same groups whether or
// not a range beside them has been rewritten; ranges are disjoint and each is
// read into registers before it is written back.  In shared memory a key is
// (group index within the range, low bits): group numbers skip the groups
// already resolved, so the range's own numbering keeps the key to 32 bits
// (else the range is left to the global passes).  Stable 8-bit passes rank
// like the global scatter (warps own consecutive elements, equal digits in
// order by __match_any_sync and per-warp running counts); the group bits
// written back are those already at each index.
constexpr int kSegThreads = 512;
constexpr int kSegWarps = kSegThreads / 32;
constexpr uint32_t kSegWin = 2048;
constexpr uint32_t kSegCap = 2 * kSegWin;
constexpr uint32_t kSegSteps = kSegCap / kSegWarps / 32;  // at most 8 warp steps per pass
constexpr size_t kSegSmem = (5 * (size_t)kSegCap + (size_t)kSegWarps * 256 + 256) * 4;

__global__ void __launch_bounds__(kSegThreads) k_seg_sort(uint64_t *key, uint32_t *val, uint32_t count,
                                                          uint32_t lo_bits, uint32_t *cov)
{
    extern __shared__ __align__(16) uint32_t seg_sm[];
    uint32_t *sk = seg_sm;                      // [2][kSegCap] range keys
    uint32_t *sv = sk + 2 * kSegCap;            // [2][kSegCap] values
    uint32_t *sg = sv + 2 * kSegCap;            // [kSegCap] group numbers of [w0, w2)
    uint32_t *wcnt = sg + kSegCap;              // [kSegWarps][256]
    uint32_t *dstart = wcnt + kSegWarps * 256;  // [256]
    __shared__ uint32_t s_a, s_b, s_l, s_gprev, s_ws[kSegWarps];
    const uint32_t tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const uint64_t w0 = (uint64_t)blockIdx.x * kSegWin;
    const uint64_t w1 = w0 + kSegWin < count ? w0 + kSegWin : count;
    const uint64_t w2 = w0 + kSegCap < count ? w0 + kSegCap : count;
    const uint32_t span = (uint32_t)(w2 - w0), win = (uint32_t)(w1 - w0);
    const uint64_t lo_mask = (1ull << lo_bits) - 1;
    // [w0, w2) into shared memory, coalesced: group numbers (they fit 32 bits:
    // fewer than count) and low bits (in the second key buffer for now)
    for (uint32_t i = tid; i < span; i += kSegThreads) {
        const uint64_t k = key[w0 + i];
        sg[i] = (uint32_t)(k >> lo_bits);
        sk[kSegCap + i] = (uint32_t)(k & lo_mask);
    }
    if (tid == 0) {
        s_a = kNil;
        s_b = kNil;
        s_l = 0;
        s_gprev = w0 > 0 ? (uint32_t)(key[w0 - 1] >> lo_bits) : kNil;
    }
    __syncthreads();
    {  // group starts in [w0, w2), one atomic per warp
        uint32_t a = kNil, l = 0, b = kNil;
        for (uint32_t i = tid; i < span; i += kSegThreads) {
            const bool st = i == 0 ? (w0 == 0 || sg[0] != s_gprev) : sg[i] != sg[i - 1];
            if (st) {
                if (i < win) {
                    a = i < a ? i : a;
                    l = i > l ? i : l;
                } else {
                    b = i < b ? i : b;
                }
            }
        }
        a = __reduce_min_sync(0xffffffffu, a);
        b = __reduce_min_sync(0xffffffffu, b);
        l = __reduce_max_sync(0xffffffffu, l);
        if (lane == 0) {
            atomicMin(&s_a, a);
            atomicMin(&s_b, b);
            atomicMax(&s_l, l);
        }
    }
    __syncthreads();
    const uint32_t a = s_a;
    if (a == kNil)
        return;  // no group starts in this window
    const uint32_t b = s_b != kNil ? s_b : (w2 == count ? span : s_l);
    if (b <= a)
        return;
    const uint32_t m = b - a;
    // warp w ranks the elements [w * steps * 32, (w + 1) * steps * 32) of the
    // range in every pass: an equal share each, in element order
    const uint32_t steps = (m + kSegThreads - 1) / kSegThreads;
    // each element's group index within the range: starts counted by ballots
    // over the warp's elements, then across the warps
    uint32_t mine = 0;
    for (uint32_t j = 0; j < steps; ++j) {
        const uint32_t i = (w * steps + j) * 32 + lane;
        const bool st = i > 0 && i < m && sg[a + i] != sg[a + i - 1];
        mine += __popc(__ballot_sync(0xffffffffu, st));
    }
    uint32_t groups;
    const uint32_t wbefore = srt::block_excl_scan(lane == 0 ? mine : 0u, s_ws, groups);
    const uint32_t wbase = __shfl_sync(0xffffffffu, wbefore, 0);
    if (((uint64_t)(groups + 1) << lo_bits) - 1 > 0xffffffffull)
        return;  // keys of this range wider than 32 bits: global passes
    const uint32_t bits = 64 - __clzll((long long)((((uint64_t)groups + 1) << lo_bits) - 1));
    {
        uint32_t run = wbase;
        for (uint32_t j = 0; j < steps; ++j) {
            const uint32_t i = (w * steps + j) * 32 + lane;
            const bool st = i > 0 && i < m && sg[a + i] != sg[a + i - 1];
            const uint32_t mask = __ballot_sync(0xffffffffu, st);
            if (i < m)
                sk[i] = ((run + __popc(mask & srt::lanemask_le())) << lo_bits) | sk[kSegCap + a + i];
            run += __popc(mask);
        }
    }
    for (uint32_t i = tid; i < m; i += kSegThreads)
        sv[i] = val[w0 + a + i];
    __syncthreads();
    uint32_t cur = 0;
    for (uint32_t shift = 0; shift < bits; shift += 8) {
        for (uint32_t i = tid; i < kSegWarps * 256; i += kSegThreads)
            wcnt[i] = 0;
        __syncthreads();
        const uint32_t *ck = sk + cur * kSegCap, *cv = sv + cur * kSegCap;
        uint32_t rank[kSegSteps], dg[kSegSteps];
#pragma unroll
        for (uint32_t j = 0; j < kSegSteps; ++j) {
            if (j >= steps)
                break;
            const uint32_t e = (w * steps + j) * 32 + lane;
            const uint32_t d = e < m ? (ck[e] >> shift) & 255u : 256u;
            const uint32_t mask = __match_any_sync(0xffffffffu, d);
            rank[j] = d < 256u ? wcnt[w * 256 + d] + __popc(mask & srt::lanemask_lt()) : 0u;
            __syncwarp();
            if (d < 256u && lane == (uint32_t)__ffs(mask) - 1)
                wcnt[w * 256 + d] += __popc(mask);
            __syncwarp();
            dg[j] = d;
        }
        __syncthreads();
        // per digit: exclusive prefix over the warps, then over the digits
        uint32_t run = 0, x = 0;
        if (tid < 256) {
#pragma unroll
            for (int ww = 0; ww < kSegWarps; ++ww) {
                const uint32_t t = wcnt[ww * 256 + tid];
                wcnt[ww * 256 + tid] = run;
                run += t;
            }
            x = run;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
                if (lane >= (uint32_t)d)
                    x += y;
            }
            if (lane == 31)
                s_ws[w] = x;
        }
        __syncthreads();
        if (tid < 256) {
            uint32_t pre = 0;
            for (uint32_t ww = 0; ww < w; ++ww)
                pre += s_ws[ww];
            dstart[tid] = pre + x - run;
        }
        __syncthreads();
        uint32_t *nk = sk + (cur ^ 1) * kSegCap, *nv = sv + (cur ^ 1) * kSegCap;
#pragma unroll
        for (uint32_t j = 0; j < kSegSteps; ++j) {
            if (j >= steps)
                break;
            const uint32_t e = (w * steps + j) * 32 + lane;
            if (dg[j] < 256u) {
                const uint32_t q = dstart[dg[j]] + wcnt[w * 256 + dg[j]] + rank[j];
                nk[q] = ck[e];
                nv[q] = cv[e];
            }
        }
        __syncthreads();
        cur ^= 1;
    }
    const uint32_t *ck = sk + cur * kSegCap, *cv = sv + cur * kSegCap;
    for (uint32_t i = tid; i < m; i += kSegThreads) {
        key[w0 + a + i] = ((uint64_t)sg[a + i] << lo_bits) | ((uint64_t)ck[i] & lo_mask);
        val[w0 + a + i] = cv[i];
        cov[w0 + a + i] = 1u;
    }
}

// flags[k] = 1 - cov[k]: the members of groups left to the global passes
__global__ void k_uncovered(uint32_t *cov, uint32_t count)
{
    for (uint32_t k = blockIdx.x * kEw + threadIdx.x; k < count; k += gridDim.x * kEw)
        cov[k] = 1u - cov[k];
}

// gather the uncovered elements (inclusive scan of their flags in incl) in
// list order, with their list indices
__global__ void k_gather_uncovered(const uint64_t *key, const uint32_t *val, const uint32_t *incl,
                                   uint32_t count, uint64_t *gk, uint32_t *gv, uint32_t *idx)
{
    for (uint32_t k = blockIdx.x * kEw + threadIdx.x; k < count; k += gridDim.x * kEw) {
        const uint32_t c = incl[k];
        if (c != (k ? incl[k - 1] : 0u)) {
            gk[c - 1] = key[k];
            gv[c - 1] = val[k];
            idx[c - 1] = k;
        }
    }
}

// the sorted uncovered elements back to their list indices: each large group
// owns the same indices before and after, so list order is kept
__global__ void k_scatter_uncovered(const uint64_t *gk, const uint32_t *gv, const uint32_t *idx,
                                    uint32_t count, uint64_t *key, uint32_t *val)
{
    for (uint32_t j = blockIdx.x * kEw + threadIdx.x; j < count; j += gridDim.x * kEw) {
        key[idx[j]] = gk[j];
        val[idx[j]] = gv[j];
    }
}

// ---- refining the groups of a sorted active list ---------------------------
// Element k of the sorted list starts a group when its key differs from
// k-1's (head), and its group has two members or more unless it is a head
// whose successor is a head too (flag).  One scan over the list gives, per
// element, the number of heads up to it (its group's number + 1), the number
// of flagged elements before it (its place in the next active list) and the
// largest head slot up to it (its group's first slot: slots increase along
// the list, so the last head wins), the three carried together.  From round 1
// on, a head that also starts a group of the round before (the key's group
// bits change there) carries a mark in the slot's low bit: elements whose
// last head is marked keep the first slot they had, so their rank is not
// written again.
constexpr int kRfThreads = 512;
constexpr int kRfItems = 8;
constexpr uint32_t kRfTile = kRfThreads * kRfItems;

struct AddOp {
    __device__ __forceinline__ uint32_t operator()(uint32_t a, uint32_t b) const { return a + b; }
};
struct MaxOp {
    __device__ __forceinline__ uint32_t operator()(uint32_t a, uint32_t b) const { return a > b ? a : b; }
};

// block-wide exclusive scan under op (kRfThreads threads), *total the
// reduction of all
template <class Op>
__device__ __forceinline__ uint32_t rf_block_scan(uint32_t v, uint32_t *ws, uint32_t &total, Op op,
                                                  uint32_t id)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d)
            x = op(x, y);
    }
    if (lane == 31)
        ws[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t t = lane < kRfThreads / 32 ? ws[lane] : id;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, t, d);
            if (lane >= d)
                t = op(t, y);
        }
        if (lane < kRfThreads / 32)
            ws[lane] = t;
    }
    __syncthreads();
    total = ws[kRfThreads / 32 - 1];
    const uint32_t before = w > 0 ? ws[w - 1] : id;
    uint32_t xe = __shfl_up_sync(0xffffffffu, x, 1);
    if (lane == 0)
        xe = id;
    __syncthreads();
    return op(before, xe);
}

struct RfItems {
    uint32_t head[kRfItems], flag[kRfItems], slot[kRfItems];
};

// A tile's keys and slots staged in shared memory with coalesced loads, so
// that each thread then reads its kRfItems consecutive elements from there.
// Index t is stored at t + t / 8: a thread's 8 consecutive words and a warp's
// consecutive fills then fall in distinct banks.
__device__ __forceinline__ uint32_t rf_pad(uint32_t t) { return t + (t >> 3); }
constexpr uint32_t kRfKeyWords = kRfTile + 2 + (kRfTile + 2) / 8 + 1;  // keys of [t0 - 1, t0 + kRfTile + 1)
constexpr uint32_t kRfIdxWords = kRfTile + kRfTile / 8;
constexpr size_t kRfTilesSmem = 8 * (size_t)kRfKeyWords + 4 * (size_t)kRfIdxWords;
constexpr size_t kRfApplySmem = kRfTilesSmem + 4 * (size_t)kRfIdxWords;

__device__ __forceinline__ void rf_stage(const uint64_t *key, const uint32_t *act, const uint32_t *val,
                                         uint32_t count, uint64_t t0, uint64_t *skey, uint32_t *sact,
                                         uint32_t *sval)
{
    for (uint32_t t = threadIdx.x; t < kRfTile + 2; t += kRfThreads) {
        const uint64_t k = t0 + t;  // element k - 1
        skey[rf_pad(t)] = (k >= 1 && k - 1 < count) ? key[k - 1] : 0ull;
    }
    for (uint32_t t = threadIdx.x; t < kRfTile; t += kRfThreads) {
        const uint64_t k = t0 + t;
        sact[rf_pad(t)] = k < count ? act[k] : 0u;
        if (val)
            sval[rf_pad(t)] = k < count ? val[k] : 0u;
    }
    __syncthreads();
}

// the values of this thread's kRfItems consecutive elements (from the stage)
__device__ __forceinline__ RfItems rf_items(const uint64_t *skey, const uint32_t *sact, uint32_t count,
                                            uint64_t t0, uint32_t gbits)
{
    const uint32_t t = threadIdx.x * kRfItems;
    const uint64_t base = t0 + t;
    uint64_t kk[kRfItems + 2];
#pragma unroll
    for (int j = 0; j < kRfItems + 2; ++j)
        kk[j] = skey[rf_pad(t + j)];  // element base + j - 1
    RfItems r;
#pragma unroll
    for (int j = 0; j < kRfItems; ++j) {
        const uint64_t k = base + j;
        const bool ok = k < count;
        const bool hd = ok && (k == 0 || kk[j + 1] != kk[j]);
        const bool nh = k + 1 >= count || kk[j + 2] != kk[j + 1];
        // gbits < 64: the key's bits from gbits up are the previous round's group
        const bool old = gbits < 64 && hd && (k == 0 || (kk[j + 1] >> gbits) != (kk[j] >> gbits));
        r.head[j] = hd ? 1u : 0u;
        r.flag[j] = (ok && !(hd && nh)) ? 1u : 0u;
        r.slot[j] = hd ? (sact[rf_pad(t + j)] << 1) | (old ? 1u : 0u) : 0u;
    }
    return r;
}

__global__ void __launch_bounds__(kRfThreads) k_refine_tiles(const uint64_t *key, const uint32_t *act,
                                                             uint32_t count, uint32_t gbits,
                                                             uint32_t *ph, uint32_t *pf, uint32_t *pm)
{
    extern __shared__ __align__(16) uint64_t rf_sm[];
    uint64_t *skey = rf_sm;
    uint32_t *sact = reinterpret_cast<uint32_t *>(rf_sm + kRfKeyWords);
    __shared__ uint32_t ws[kRfThreads / 32];
    const uint64_t t0 = (uint64_t)blockIdx.x * kRfTile;
    rf_stage(key, act, nullptr, count, t0, skey, sact, nullptr);
    const RfItems r = rf_items(skey, sact, count, t0, gbits);
    uint32_t h = 0, f = 0, m = 0;
#pragma unroll
    for (int j = 0; j < kRfItems; ++j) {
        h += r.head[j];
        f += r.flag[j];
        m = r.slot[j] > m ? r.slot[j] : m;
    }
    uint32_t th, tf, tm;
    rf_block_scan(h, ws, th, AddOp(), 0u);
    rf_block_scan(f, ws, tf, AddOp(), 0u);
    rf_block_scan(m, ws, tm, MaxOp(), 0u);
    if (threadIdx.x == 0) {
        ph[blockIdx.x] = th;
        pf[blockIdx.x] = tf;
        pm[blockIdx.x] = tm;
    }
}

// one CTA: exclusive scans of the tile aggregates in place; the totals of
// heads (groups) and flags (next active count) to tot[0], tot[1]
__global__ void __launch_bounds__(kRfThreads) k_refine_parts(uint32_t *ph, uint32_t *pf, uint32_t *pm,
                                                             uint32_t tiles, uint32_t *tot)
{
    __shared__ uint32_t ws[kRfThreads / 32];
    uint32_t ch = 0, cf = 0, cm = 0;
    for (uint32_t b = 0; b < tiles; b += kRfThreads) {
        const uint32_t i = b + threadIdx.x;
        const bool ok = i < tiles;
        uint32_t th, tf, tm;
        const uint32_t xh = rf_block_scan(ok ? ph[i] : 0u, ws, th, AddOp(), 0u);
        const uint32_t xf = rf_block_scan(ok ? pf[i] : 0u, ws, tf, AddOp(), 0u);
        const uint32_t xm = rf_block_scan(ok ? pm[i] : 0u, ws, tm, MaxOp(), 0u);
        if (ok) {
            ph[i] = ch + xh;
            pf[i] = cf + xf;
            pm[i] = xm > cm ? xm : cm;
        }
        ch += th;
        cf += tf;
        cm = tm > cm ? tm : cm;
    }
    if (threadIdx.x == 0) {
        tot[0] = ch;
        tot[1] = cf;
    }
}

// sorted slots back into SA, new ranks scattered to the positions, and the
// elements of groups still unresolved appended to the next active list with
// their group numbers (staged in shared memory, where the keys were, and
// written out coalesced)
__global__ void __launch_bounds__(kRfThreads) k_refine_apply(
    const uint64_t *key, const uint32_t *val, const uint32_t *act, uint32_t count, uint32_t gbits,
    const uint32_t *ph, const uint32_t *pf, const uint32_t *pm, uint32_t *sa, uint32_t *rk,
    uint32_t *act2, uint32_t *grp2)
{
    extern __shared__ __align__(16) uint64_t rf_sm[];
    uint64_t *skey = rf_sm;
    uint32_t *sact = reinterpret_cast<uint32_t *>(rf_sm + kRfKeyWords);
    uint32_t *sval = sact + kRfIdxWords;
    uint32_t *so_act = reinterpret_cast<uint32_t *>(rf_sm);  // after the keys are read
    uint32_t *so_grp = so_act + kRfIdxWords;
    __shared__ uint32_t ws[kRfThreads / 32];
    const uint64_t t0 = (uint64_t)blockIdx.x * kRfTile;
    rf_stage(key, act, val, count, t0, skey, sact, sval);
    for (uint32_t t = threadIdx.x; t < kRfTile && t0 + t < count; t += kRfThreads)
        sa[sact[rf_pad(t)]] = sval[rf_pad(t)];
    const RfItems r = rf_items(skey, sact, count, t0, gbits);
    uint32_t h = 0, f = 0, m = 0;
#pragma unroll
    for (int j = 0; j < kRfItems; ++j) {
        h += r.head[j];
        f += r.flag[j];
        m = r.slot[j] > m ? r.slot[j] : m;
    }
    uint32_t th, tf, tm;
    uint32_t gh = ph[blockIdx.x] + rf_block_scan(h, ws, th, AddOp(), 0u);
    uint32_t lf = rf_block_scan(f, ws, tf, AddOp(), 0u);  // flagged before, within the tile
    const uint32_t xm = rf_block_scan(m, ws, tm, MaxOp(), 0u);  // (its barriers: keys all read)
    const uint32_t pmb = pm[blockIdx.x];
    uint32_t gm = xm > pmb ? xm : pmb;
    const uint32_t t = threadIdx.x * kRfItems;
#pragma unroll
    for (int j = 0; j < kRfItems; ++j) {
        if (t0 + t + j >= count)
            break;
        gh += r.head[j];
        gm = r.slot[j] > gm ? r.slot[j] : gm;
        if (!(gm & 1u))  // else the group's first slot is unchanged
            rk[sval[rf_pad(t + j)]] = gm >> 1;
        if (r.flag[j]) {
            so_act[rf_pad(lf)] = sact[rf_pad(t + j)];
            so_grp[rf_pad(lf)] = gh - 1;
        }
        lf += r.flag[j];
    }
    __syncthreads();
    const uint32_t pfb = pf[blockIdx.x];
    for (uint32_t i = threadIdx.x; i < tf; i += kRfThreads) {
        act2[pfb + i] = so_act[rf_pad(i)];
        grp2[pfb + i] = so_grp[rf_pad(i)];
    }
}

__global__ void k_bwt_output(const uint8_t *x, const uint32_t *sa, uint32_t n, uint32_t block,
                             uint8_t *last, uint32_t *primary)
{
    for (uint32_t p = blockIdx.x * kEw + threadIdx.x; p < n; p += gridDim.x * kEw) {
        const uint32_t i = sa[p];
        uint32_t s, m;
        block_span(p, block, n, s, m);
        last[p] = x[i == s ? s + m - 1 : i - 1];
        if (i == s)
            primary[p / block] = p - s;
    }
}

struct FwdWs {
    uint32_t *sa, *rk, *act, *act2, *grp, *grp2, *part, *scal;
    uint64_t *k0, *k1;
    uint32_t *v0, *v1;
    void *radix;
    uint64_t bytes;
};

template <class T>
T *carve(uint8_t *base, uint64_t &off, uint64_t bytes)
{
    T *p = reinterpret_cast<T *>(base ? base + off : nullptr);
    off += (bytes + 255) & ~255ull;
    return p;
}

FwdWs fwd_layout(uint8_t *base, uint64_t n)
{
    FwdWs w;
    uint64_t off = 0;
    w.sa = carve<uint32_t>(base, off, 4 * n);
    w.rk = carve<uint32_t>(base, off, 4 * n);
    w.act = carve<uint32_t>(base, off, 4 * n);
    w.act2 = carve<uint32_t>(base, off, 4 * n);
    w.grp = carve<uint32_t>(base, off, 4 * n);
    w.grp2 = carve<uint32_t>(base, off, 4 * n);
    w.part = carve<uint32_t>(base, off, 3 * 4 * (uint64_t)div_up(n, kRfTile) + 16);
    w.scal = carve<uint32_t>(base, off, 16);
    w.k0 = carve<uint64_t>(base, off, 8 * n);
    w.k1 = carve<uint64_t>(base, off, 8 * n);
    w.v0 = carve<uint32_t>(base, off, 4 * n);
    w.v1 = carve<uint32_t>(base, off, 4 * n);
    w.radix = carve<uint8_t>(base, off, radix_scratch_bytes(n));
    w.bytes = off;
    return w;
}

// stable LSD over the key bits [0, bits)
cudaError_t sort_keys(FwdWs &w, uint32_t count, uint32_t bits, cudaStream_t s, uint64_t *&ks,
                      uint32_t *&vs)
{
    bool f = false;
    const cudaError_t e = radix_sort_bits(w.k0, w.v0, w.k1, w.v1, count, 0, bits, w.radix, s, f);
    ks = f ? w.k1 : w.k0;
    vs = f ? w.v1 : w.v0;
    return e;
}

// sort a round's active list (keys in k0/v0, already in group order) by its
// key bits [0, bits): small groups in shared memory in place, the members of
// the others gathered into k1/v1 (the second half as the ping-pong buffer),
// sorted by the global passes and put back.  If they are more than half the
// list, the whole list takes the global passes.  act2 / grp2 are free until
// the refinement and hold the indices and flags.
cudaError_t sort_groups(FwdWs &w, uint32_t count, uint32_t lo_bits, uint32_t bits, cudaStream_t s,
                        uint64_t *&ks, uint32_t *&vs)
{
    static KernelSetup setup;
    int per_sm = 0;
    cudaError_t e = kernel_setup(setup, (const void *)k_seg_sort, kSegThreads, kSegSmem, &per_sm);
    if (e != cudaSuccess)
        return e;
    uint32_t *cov = w.grp2, *idx = w.act2;
    if ((e = cudaMemsetAsync(cov, 0, 4ull * count, s)) != cudaSuccess)
        return e;
    k_seg_sort<<<div_up(count, kSegWin), kSegThreads, kSegSmem, s>>>(w.k0, w.v0, count, lo_bits, cov);
    k_uncovered<<<ew_grid(count), kEw, 0, s>>>(cov, count);
    if ((e = scan_u32(cov, cov, count, true, w.part, w.scal + 2, s)) != cudaSuccess)
        return e;
    uint32_t big = 0;
    if ((e = cudaMemcpyAsync(&big, w.scal + 2, sizeof(big), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return e;
    ks = w.k0;
    vs = w.v0;
    if (big == 0)
        return cudaSuccess;
    if (2ull * big > count)
        return sort_keys(w, count, bits, s, ks, vs);
    k_gather_uncovered<<<ew_grid(count), kEw, 0, s>>>(w.k0, w.v0, cov, count, w.k1, w.v1, idx);
    bool f = false;
    if ((e = radix_sort_bits(w.k1, w.v1, w.k1 + big, w.v1 + big, big, 0, bits, w.radix, s, f)) !=
        cudaSuccess)
        return e;
    k_scatter_uncovered<<<ew_grid(big), kEw, 0, s>>>(f ? w.k1 + big : w.k1, f ? w.v1 + big : w.v1,
                                                      idx, big, w.k0, w.v0);
    return cudaGetLastError();
}

// split the groups of the sorted active list; returns the number still
// unresolved and the number of groups of the list (host values)
cudaError_t refine(FwdWs &w, const uint64_t *ks, const uint32_t *vs, uint32_t count,
                   uint32_t gbits, cudaStream_t s, uint32_t &n_act, uint32_t &groups)
{
    const uint32_t tiles = div_up(count, kRfTile);
    uint32_t *ph = w.part, *pf = w.part + tiles, *pm = w.part + 2 * tiles;
    static KernelSetup setup_tiles, setup_apply;
    int per_sm = 0;
    cudaError_t e;
    if ((e = kernel_setup(setup_tiles, (const void *)k_refine_tiles, kRfThreads, kRfTilesSmem,
                          &per_sm)) != cudaSuccess ||
        (e = kernel_setup(setup_apply, (const void *)k_refine_apply, kRfThreads, kRfApplySmem,
                          &per_sm)) != cudaSuccess)
        return e;
    k_refine_tiles<<<tiles, kRfThreads, kRfTilesSmem, s>>>(ks, w.act, count, gbits, ph, pf, pm);
    k_refine_parts<<<1, kRfThreads, 0, s>>>(ph, pf, pm, tiles, w.scal);
    k_refine_apply<<<tiles, kRfThreads, kRfApplySmem, s>>>(ks, vs, w.act, count, gbits, ph, pf, pm,
                                                           w.sa, w.rk, w.act2, w.grp2);
    uint32_t h[2];
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpyAsync(h, w.scal, sizeof(h), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return e;
    groups = h[0];
    n_act = h[1];
    uint32_t *t = w.act;
    w.act = w.act2;
    w.act2 = t;
    t = w.grp;
    w.grp = w.grp2;
    w.grp2 = t;
    return cudaSuccess;
}

// ---- inverse --------------------------------------------------------------
__global__ void k_lf_keys(const uint8_t *last, uint32_t n, uint32_t block, uint64_t *key,
                          uint32_t *val)
{
    for (uint32_t p = blockIdx.x * kEw + threadIdx.x; p < n; p += gridDim.x * kEw) {
        key[p] = ((uint64_t)(p / block) << 8) | last[p];
        val[p] = p;
    }
}

__global__ void k_lf_scatter(const uint32_t *vs, uint32_t n, uint32_t *lf)
{
    for (uint32_t q = blockIdx.x * kEw + threadIdx.x; q < n; q += gridDim.x * kEw)
        lf[vs[q]] = q;
}

__global__ void k_check_primary(const uint32_t *primary, uint32_t n, uint32_t block,
                                uint32_t blocks, int32_t *status)
{
    for (uint32_t b = blockIdx.x * kEw + threadIdx.x; b < blocks; b += gridDim.x * kEw) {
        const uint32_t s = b * block;
        const uint32_t m = n - s < block ? n - s : block;
        if (primary[b] >= m)
            set_status(status, HUFF_ERR_CORRUPT_STREAM);
    }
}

struct Samples {
    uint32_t n, block, regular;  // regular samples: rows 0, 64, 128, ...
    const uint32_t *primary;
    // sample id of row p, or kNil: a primary row is its block's extra
    // sample (regular + block), even when it is also a multiple of 64
    __device__ __forceinline__ uint32_t id_of(uint32_t p) const
    {
        const uint32_t b = p / block;
        if (p - b * block == primary[b])
            return regular + b;
        return (p % kSampleGap) == 0 ? p / kSampleGap : kNil;
    }
    // row of sample id, or kNil for a regular sample that is a primary row
    __device__ __forceinline__ uint32_t row_of(uint32_t id) const
    {
        if (id >= regular)
            return (id - regular) * block + primary[id - regular];
        const uint32_t p = id * kSampleGap;
        const uint32_t b = p / block;
        return p - b * block == primary[b] ? kNil : p;
    }
};

// every sample walks to the next sample: link and length; the link into a
// block's primary sample is cut (kNil), which turns the primary's cycle into
// a list headed by the primary
__global__ void k_walk_link(const uint32_t *lf, Samples S, uint32_t count, uint32_t *nxt,
                            uint32_t *len, int32_t *status)
{
    if (chain_failed(status))
        return;
    for (uint32_t id = blockIdx.x * kEw + threadIdx.x; id < count; id += gridDim.x * kEw) {
        const uint32_t p0 = S.row_of(id);
        if (p0 == kNil) {
            nxt[id] = kNil;
            len[id] = 0;
            continue;
        }
        uint32_t s, m;
        block_span(p0, S.block, S.n, s, m);
        uint32_t p = p0, t = 0, c;
        do {  // ends on p0 at the latest: LF is a permutation of the block
            p = lf[p];
            ++t;
            c = p < S.n ? S.id_of(p) : kNil;
        } while (c == kNil && t < m && p < S.n);
        if (c == kNil) {  // not a permutation: cannot happen for a sorted column
            set_status(status, HUFF_ERR_CORRUPT_STREAM);
            nxt[id] = kNil;
            len[id] = 0;
            continue;
        }
        const uint32_t b = p0 / S.block;
        nxt[id] = c == S.regular + b ? kNil : c;
        len[id] = t;
    }
}

// one pointer-jumping step: sum[id] = stretch lengths from id to the list's
// end after enough steps
__global__ void k_jump(const uint32_t *nx_in, const uint32_t *sum_in, uint32_t count,
                       uint32_t *nx_out, uint32_t *sum_out, const int32_t *status)
{
    if (chain_failed(status))
        return;
    for (uint32_t id = blockIdx.x * kEw + threadIdx.x; id < count; id += gridDim.x * kEw) {
        const uint32_t x = nx_in[id];
        if (x == kNil) {
            nx_out[id] = kNil;
            sum_out[id] = sum_in[id];
        } else {
            nx_out[id] = nx_in[x];
            sum_out[id] = sum_in[id] + sum_in[x];
        }
    }
}

// samples on their block's primary list write their stretch: the primary's
// sum is the cycle length c, a sample's distance from the primary is
// c - its own sum
__global__ void k_walk_emit(const uint32_t *lf, const uint8_t *last, Samples S, uint32_t count,
                            const uint32_t *len, const uint32_t *nx, const uint32_t *sum,
                            uint8_t *out, int32_t *status)
{
    if (chain_failed(status))
        return;
    for (uint32_t id = blockIdx.x * kEw + threadIdx.x; id < count; id += gridDim.x * kEw) {
        const uint32_t L = len[id];
        if (L == 0 || nx[id] != kNil)
            continue;  // not a sample, or not on the primary's cycle
        uint32_t p = S.row_of(id);
        uint32_t s, m;
        block_span(p, S.block, S.n, s, m);
        const uint32_t c = sum[S.regular + p / S.block];
        const uint32_t d = c - sum[id];
        if (c > m || d + L > c) {
            set_status(status, HUFF_ERR_CORRUPT_STREAM);
            continue;
        }
        for (uint32_t t = 0; t < L && p < S.n; ++t) {
            out[s + m - 1 - (d + t)] = last[p];
            p = lf[p];
        }
    }
}

// a block whose walk closed after c < m rows repeats its last c bytes
__global__ void k_periodic_fill(uint8_t *out, uint32_t n, uint32_t block, uint32_t regular,
                                const uint32_t *sum, const int32_t *status)
{
    if (chain_failed(status))
        return;
    for (uint32_t q = blockIdx.x * kEw + threadIdx.x; q < n; q += gridDim.x * kEw) {
        uint32_t s, m;
        block_span(q, block, n, s, m);
        const uint32_t c = sum[regular + q / block];
        const uint32_t t = s + m - 1 - q;  // walk step of q
        if (c < m && t >= c)
            out[q] = out[s + m - 1 - t % c];
    }
}

struct InvWs {
    uint32_t *lf, *nxt, *len, *nx2, *sum, *sum2;
    uint64_t *k0, *k1;
    uint32_t *v0, *v1;
    void *radix;
    uint64_t bytes;
};

uint32_t sample_count(uint64_t n, uint32_t block)
{
    return (uint32_t)((n + kSampleGap - 1) / kSampleGap + (n + block - 1) / block);
}

InvWs inv_layout(uint8_t *base, uint64_t n, uint32_t block)
{
    InvWs w;
    uint64_t off = 0;
    const uint64_t S = sample_count(n, block);
    w.lf = carve<uint32_t>(base, off, 4 * n);
    w.nxt = carve<uint32_t>(base, off, 4 * S);
    w.len = carve<uint32_t>(base, off, 4 * S);
    w.nx2 = carve<uint32_t>(base, off, 4 * S);
    w.sum = carve<uint32_t>(base, off, 4 * S);
    w.sum2 = carve<uint32_t>(base, off, 4 * S);
    w.k0 = carve<uint64_t>(base, off, 8 * n);
    w.k1 = carve<uint64_t>(base, off, 8 * n);
    w.v0 = carve<uint32_t>(base, off, 4 * n);
    w.v1 = carve<uint32_t>(base, off, 4 * n);
    w.radix = carve<uint8_t>(base, off, radix_scratch_bytes(n));
    w.bytes = off;
    return w;
}

bool bwt_args_ok(uint64_t n, uint32_t block)
{
    return block >= 1 && n <= HUFF_BWT_MAX_N;
}

inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

__global__ void k_m3_header(uint8_t *out, uint64_t n, uint32_t block, uint32_t count,
                            uint32_t stages, uint32_t head)
{
    for (uint32_t i = threadIdx.x; i < head; i += blockDim.x) {
        if (i < 8)
            out[i] = (uint8_t)(n >> (8 * i));
        else if (i < 12)
            out[i] = (uint8_t)(block >> (8 * (i - 8)));
        else if (i < 16)
            out[i] = (uint8_t)(count >> (8 * (i - 12)));
        else if (i < 20)
            out[i] = (uint8_t)(stages >> (8 * (i - 16)));
        else if (i >= 20 + 4 * count)
            out[i] = 0;
    }
}

__global__ void k_add_u64(unsigned long long *p, uint64_t v, const int32_t *status)
{
    if (!chain_failed(status))
        *p += v;
}

uint32_t m3_head_bytes(uint64_t count) { return (uint32_t)((20 + 4 * count + 15) & ~15ull); }

uint64_t max3(uint64_t a, uint64_t b, uint64_t c) { return a > b ? (a > c ? a : c) : (b > c ? b : c); }

}  // namespace
}  // namespace huff

using namespace huff;

extern "C" {

uint64_t huff_bwt_workspace_size(uint64_t n, uint32_t block)
{
    if (!bwt_args_ok(n, block))
        return 0;
    const uint64_t f = fwd_layout(nullptr, n).bytes;
    const uint64_t i = inv_layout(nullptr, n, block).bytes;
    return f > i ? f : i;
}

huff_status_t huff_bwt_forward(const uint8_t *d_in, uint64_t n, uint32_t block, uint8_t *d_last,
                               uint32_t *d_primary, void *d_ws, uint64_t ws_bytes,
                               int32_t *d_status, huff_stream_t stream)
{
    HUFF_API_RANGE("huff_bwt_forward");
    if (!bwt_args_ok(n, block) || !d_status || (n && (!d_in || !d_last || !d_primary || !d_ws)) ||
        (n && ws_bytes < huff_bwt_workspace_size(n, block)) || (d_ws && !aligned16(d_ws)))
        return HUFF_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(d_status, 0, sizeof(int32_t), s) != cudaSuccess)
        return HUFF_ERR_CUDA;
    if (n == 0)
        return HUFF_OK;
    const uint32_t N = (uint32_t)n;
    FwdWs w = fwd_layout(static_cast<uint8_t *>(d_ws), n);
    const uint64_t blocks = (n + block - 1) / block;
    const uint64_t mmax = n < block ? n : block;
    k_bwt_init<<<ew_grid(n), kEw, 0, s>>>(d_in, N, block, w.k0, w.v0, w.act);
    uint64_t *ks;
    uint32_t *vs;
    if (sort_keys(w, N, 32 + bit_width(blocks - 1), s, ks, vs) != cudaSuccess)
        return HUFF_ERR_CUDA;
    uint32_t n_act = 0, groups = 0;
    if (refine(w, ks, vs, N, 64, s, n_act, groups) != cudaSuccess)
        return HUFF_ERR_CUDA;
    for (uint64_t h = 4; n_act > 0 && h < mmax; h *= 2) {
        const uint32_t lo_bits = bit_width(mmax - 1);
        k_bwt_round_keys<<<ew_grid(n_act), kEw, 0, s>>>(w.sa, w.rk, w.act, w.grp, n_act, N, block, h,
                                                        lo_bits, w.k0, w.v0);
        if (sort_groups(w, n_act, lo_bits, lo_bits + bit_width(groups - 1), s, ks, vs) != cudaSuccess)
            return HUFF_ERR_CUDA;
        if (refine(w, ks, vs, n_act, lo_bits, s, n_act, groups) != cudaSuccess)
            return HUFF_ERR_CUDA;
    }
    k_bwt_output<<<ew_grid(n), kEw, 0, s>>>(d_in, w.sa, N, block, d_last, d_primary);
    return cudaGetLastError() == cudaSuccess ? HUFF_OK : HUFF_ERR_CUDA;
}

huff_status_t huff_bwt_inverse(const uint8_t *d_last, uint64_t n, uint32_t block,
                               const uint32_t *d_primary, uint8_t *d_out, void *d_ws,
                               uint64_t ws_bytes, int32_t *d_status, huff_stream_t stream)
{
    HUFF_API_RANGE("huff_bwt_inverse");
    if (!bwt_args_ok(n, block) || !d_status || (n && (!d_last || !d_primary || !d_out || !d_ws)) ||
        (n && ws_bytes < huff_bwt_workspace_size(n, block)) || (d_ws && !aligned16(d_ws)))
        return HUFF_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(d_status, 0, sizeof(int32_t), s) != cudaSuccess)
        return HUFF_ERR_CUDA;
    if (n == 0)
        return HUFF_OK;
    const uint32_t N = (uint32_t)n;
    InvWs w = inv_layout(static_cast<uint8_t *>(d_ws), n, block);
    const uint32_t blocks = (uint32_t)((n + block - 1) / block);
    k_check_primary<<<ew_grid(blocks), kEw, 0, s>>>(d_primary, N, block, blocks, d_status);
    k_lf_keys<<<ew_grid(n), kEw, 0, s>>>(d_last, N, block, w.k0, w.v0);
    bool flip = false;
    if (radix_sort_bits(w.k0, w.v0, w.k1, w.v1, N, 0, 8 + bit_width(blocks - 1), w.radix, s, flip) !=
        cudaSuccess)
        return HUFF_ERR_CUDA;
    k_lf_scatter<<<ew_grid(n), kEw, 0, s>>>(flip ? w.v1 : w.v0, N, w.lf);
    Samples S;
    S.n = N;
    S.block = block;
    S.regular = (uint32_t)((n + kSampleGap - 1) / kSampleGap);
    S.primary = d_primary;
    const uint32_t count = sample_count(n, block);
    k_walk_link<<<ew_grid(count), kEw, 0, s>>>(w.lf, S, count, w.nxt, w.len, d_status);
    // the longest list is one block's samples
    const uint64_t per_block = (uint64_t)((n < block ? n : block) + kSampleGap - 1) / kSampleGap + 1;
    const uint32_t rounds = bit_width(per_block) + 1;
    uint32_t *nx = w.nxt, *sm = w.len, *nx_o = w.nx2, *sm_o = w.sum;
    for (uint32_t r = 0; r < rounds; ++r) {
        k_jump<<<ew_grid(count), kEw, 0, s>>>(nx, sm, count, nx_o, sm_o, d_status);
        if (r == 0) {  // len stays; later steps ping-pong between sum and sum2
            nx = nx_o;
            sm = sm_o;
            nx_o = w.nxt;
            sm_o = w.sum2;
        } else {
            uint32_t *t = nx;
            nx = nx_o;
            nx_o = t;
            t = sm;
            sm = sm_o;
            sm_o = t;
        }
    }
    k_walk_emit<<<ew_grid(count), kEw, 0, s>>>(w.lf, d_last, S, count, w.len, nx, sm, d_out,
                                              d_status);
    k_periodic_fill<<<ew_grid(n), kEw, 0, s>>>(d_out, N, block, S.regular, sm, d_status);
    return cudaGetLastError() == cudaSuccess ? HUFF_OK : HUFF_ERR_CUDA;
}

uint64_t huff_m3_max_size(uint64_t n, uint32_t block, uint64_t segment_bytes,
                          uint32_t chunk_symbols)
{
    if (!bwt_args_ok(n, block))
        return 0;
    const uint64_t seg = huff_segmented_max_size(n, segment_bytes, chunk_symbols);
    return seg ? m3_head_bytes((n + block - 1) / block) + seg : 0;
}

uint64_t huff_m3_workspace_size(uint64_t n, uint32_t block, uint64_t segment_bytes,
                                uint32_t chunk_symbols)
{
    if (!bwt_args_ok(n, block))
        return 0;
    const uint64_t seg = huff_segmented_workspace_size(n, segment_bytes, chunk_symbols);
    if (!seg)
        return 0;
    return ((n + 255) & ~255ull) +
           max3(huff_bwt_workspace_size(n, block), seg, huff_mtf_workspace_size(n, block));
}

huff_status_t huff_m3_compress(const uint8_t *d_in, uint64_t n, uint32_t block,
                               uint64_t segment_bytes, uint32_t chunk_symbols, uint32_t stages,
                               uint8_t *d_out, uint64_t out_cap, uint64_t *d_out_bytes,
                               void *d_ws, uint64_t ws_bytes, int32_t *d_status,
                               huff_stream_t stream)
{
    HUFF_API_RANGE("huff_m3_compress");
    const uint64_t need = huff_m3_workspace_size(n, block, segment_bytes, chunk_symbols);
    const uint64_t count = block ? (n + block - 1) / block : 0;
    const uint32_t head = m3_head_bytes(count);
    if (!need || !d_out || !d_out_bytes || !d_status || !d_ws || ws_bytes < need ||
        out_cap < head || (n && !d_in) || !aligned16(d_out) || !aligned16(d_ws) ||
        (stages & ~HUFF_M3_MTF))
        return HUFF_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    uint8_t *ws = static_cast<uint8_t *>(d_ws);
    uint8_t *last = ws;
    uint8_t *rest = ws + ((n + 255) & ~255ull);
    const uint64_t rest_bytes = ws_bytes - (uint64_t)(rest - ws);
    huff_status_t st = huff_bwt_forward(d_in, n, block, last,
                                        reinterpret_cast<uint32_t *>(d_out + 20), rest, rest_bytes,
                                        d_status, stream);
    if (st == HUFF_OK && (stages & HUFF_M3_MTF))
        st = huff_mtf_forward(last, n, block, last, rest, rest_bytes, stream);
    if (st != HUFF_OK)
        return st;
    k_m3_header<<<1, 256, 0, s>>>(d_out, n, block, (uint32_t)count, stages, head);
    if (cudaGetLastError() != cudaSuccess)
        return HUFF_ERR_CUDA;
    st = huff_segmented_compress(last, n, segment_bytes, chunk_symbols, d_out + head,
                                 out_cap - head, d_out_bytes, rest, ws_bytes - (uint64_t)(rest - ws),
                                 d_status, stream);
    if (st != HUFF_OK)
        return st;
    k_add_u64<<<1, 1, 0, s>>>(reinterpret_cast<unsigned long long *>(d_out_bytes), head, d_status);
    return cudaGetLastError() == cudaSuccess ? HUFF_OK : HUFF_ERR_CUDA;
}

uint64_t huff_m3_decompress_workspace_size(uint64_t n, uint32_t block)
{
    if (!bwt_args_ok(n, block))
        return 0;
    const uint64_t b = huff_bwt_workspace_size(n, block), m = huff_mtf_workspace_size(n, block);
    return ((n + 255) & ~255ull) + (b > m ? b : m);
}

huff_status_t huff_m3_decompress(const uint8_t *d_in, uint64_t in_bytes, uint8_t *d_out,
                                 uint64_t out_cap, uint64_t *d_n, void *d_ws, uint64_t ws_bytes,
                                 int32_t *d_status, huff_stream_t stream)
{
    HUFF_API_RANGE("huff_m3_decompress");
    if (!d_in || !d_n || !d_status || !aligned16(d_in) || (d_ws && !aligned16(d_ws)))
        return HUFF_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(d_status, 0, sizeof(int32_t), s) != cudaSuccess)
        return HUFF_ERR_CUDA;
    uint8_t h[20];
    uint64_t n = 0;
    uint32_t block = 0, count = 0, stages = 0;
    bool ok = in_bytes >= 20;
    if (ok) {
        if (cudaMemcpyAsync(h, d_in, 20, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return HUFF_ERR_CUDA;
        for (int i = 7; i >= 0; --i)
            n = (n << 8) | h[i];
        for (int i = 11; i >= 8; --i)
            block = (block << 8) | h[i];
        for (int i = 15; i >= 12; --i)
            count = (count << 8) | h[i];
        for (int i = 19; i >= 16; --i)
            stages = (stages << 8) | h[i];
        ok = block >= 1 && n <= HUFF_BWT_MAX_N && count == (n + block - 1) / block &&
             (stages & ~HUFF_M3_MTF) == 0 && 20 + 4ull * count <= in_bytes &&
             m3_head_bytes(count) <= in_bytes;
    }
    if (!ok) {
        static const int32_t corrupt = HUFF_ERR_CORRUPT_STREAM;
        if (cudaMemcpyAsync(d_status, &corrupt, 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return HUFF_ERR_CUDA;
        return HUFF_OK;
    }
    if (n > out_cap) {
        static const int32_t cap = HUFF_ERR_CAPACITY;
        if (cudaMemcpyAsync(d_status, &cap, 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return HUFF_ERR_CUDA;
        return HUFF_OK;
    }
    if (!d_out || !d_ws || ws_bytes < huff_m3_decompress_workspace_size(n, block))
        return HUFF_ERR_INVALID_ARG;
    const uint32_t head = m3_head_bytes(count);
    uint8_t *ws = static_cast<uint8_t *>(d_ws);
    uint8_t *last = ws;
    uint8_t *rest = ws + ((n + 255) & ~255ull);
    huff_status_t st = huff_segmented_decompress(d_in + head, in_bytes - head, last, n, d_n,
                                                 d_status, stream);
    if (st != HUFF_OK)
        return st;
    // the segmented container must hold exactly n bytes
    uint64_t got = 0;
    int32_t sst = 0;
    if (cudaMemcpyAsync(&got, d_n, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&sst, d_status, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return HUFF_ERR_CUDA;
    if (sst != 0)
        return HUFF_OK;  // the segment error stays in *d_status
    if (got != n) {
        static const int32_t corrupt = HUFF_ERR_CORRUPT_STREAM;
        if (cudaMemcpyAsync(d_status, &corrupt, 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return HUFF_ERR_CUDA;
        return HUFF_OK;
    }
    const uint64_t rest_bytes = ws_bytes - (uint64_t)(rest - ws);
    if (stages & HUFF_M3_MTF) {
        st = huff_mtf_inverse(last, n, block, last, rest, rest_bytes, stream);
        if (st != HUFF_OK)
            return st;
    }
    return huff_bwt_inverse(last, n, block, reinterpret_cast<const uint32_t *>(d_in + 20), d_out,
                            rest, rest_bytes, d_status, stream);
}

}  // extern "C"
