// Batched engine: many independent buffers, each with its own codebook (the
// paper's Method 2, Section III-A, where every segment is compressed with
// its own tree and reassembled by id), compressed or decompressed in one
// persistent fused launch, captured once in a CUDA graph.
//
// One cooperative kernel (all CTAs resident) walks through phases separated
// by a software grid barrier with a bounded wait:
//   compress:   1. per-unit histograms of every 16 KiB unit of every buffer
//                  (static round robin, next unit loaded ahead);
//               2. per buffer (dynamic tickets): sum its unit histograms,
//                  build the codebook, dot each unit's histogram with the
//                  code lengths, scan them into unit bit offsets, write the
//                  stream header and size;
//               3. encode items of up to 8 units of one buffer (one unit per
//                  warp, dynamic tickets), the CTA's code table rebuilt only
//                  when the item's buffer changes.
//   decompress: 1. per buffer: read n and the chunk size from the header and
//                  size its work (chunks split across lanes so that even a
//                  one-chunk buffer fills a warp);
//               2. one CTA scans the work sizes;
//               3. decode items of up to 8 warp tasks of one buffer (dynamic
//                  tickets), tables rebuilt only when the buffer changes.
// Every step reuses the single-stream device routines (*_impl.cuh), so a
// buffer's stream is byte-identical to huff_compress on it alone.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "api_trace.h"
#include "batch_internal.cuh"
#include "codebook_impl.cuh"
#include "decode_impl.cuh"
#include "encode_impl.cuh"
#include "hist_impl.cuh"

namespace huff {
namespace {

// Sense-free generation barrier over all CTAs of a cooperative launch.
// Returns false (uniformly) when a wait gave up.
__device__ bool grid_barrier(unsigned int *ctl, int32_t *fail, uint32_t extra)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int *gen = ctl + kCtlGen;
        const unsigned int g = *gen;
        __threadfence();
        const unsigned int arrived = atomicAdd(ctl + kCtlArrive, 1u) + 1;
        int ok = 1;
        if (arrived == gridDim.x + extra) {
            ctl[kCtlArrive] = 0;
            __threadfence();
            atomicAdd(ctl + kCtlGen, 1u);
        } else {
            uint32_t spins = 0;
            while (*gen == g) {
                if (++spins > kSpinLimit || *reinterpret_cast<volatile int32_t *>(fail)) {
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        if (!ok)
            atomicCAS(fail, 0, HUFF_ERR_TIMEOUT);
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// After a barrier gave up: every buffer reports the timeout.
__device__ void fail_all(const BatchBuf *bufs, uint32_t count)
{
    if (threadIdx.x == 0)
        for (uint32_t b = 0; b < count; ++b)
            set_status(bufs[b].status, HUFF_ERR_TIMEOUT);
}


// Largest b with base[b] <= x, for x < base[count].
__device__ __forceinline__ uint32_t find_owner(const uint64_t *base, uint32_t count, uint64_t x)
{
    uint32_t lo = 0, hi = count - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (base[mid] <= x)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// The first input byte of a unit from its owner entry.
__device__ __forceinline__ const uint8_t *unit_ptr(uint4 o)
{
    return reinterpret_cast<const uint8_t *>((uint64_t)o.x | ((uint64_t)o.y << 32));
}

// A status word read once by thread 0 and broadcast, so that every thread of
// the CTA takes the same branch even while other CTAs may be setting it.
__device__ __forceinline__ bool uniform_failed(const int32_t *status)
{
    __shared__ int s_f;
    if (threadIdx.x == 0)
        s_f = chain_failed(status);
    __syncthreads();
    const bool f = s_f != 0;
    __syncthreads();
    return f;
}

__device__ __forceinline__ unsigned int take_ticket(unsigned int *ctl, int phase)
{
    __shared__ unsigned int s_t;
    if (threadIdx.x == 0)
        s_t = atomicAdd(ctl + kCtlTicket0 + phase, 1u);
    __syncthreads();
    const unsigned int t = s_t;
    __syncthreads();
    return t;
}

// Thread 0's value of t, for every thread of the CTA (a CTA barrier first,
// so it also ends the work of the item before).
__device__ __forceinline__ unsigned int cta_broadcast(unsigned int t)
{
    __shared__ unsigned int s_b;
    __syncthreads();
    if (threadIdx.x == 0)
        s_b = t;
    __syncthreads();
    return s_b;
}

// Tickets of the work loops below.  While more than a wave of items (one
// per worker: a CTA or a half) lies beyond the current one, the leader takes
// its next ticket when an item starts, so that the atomic's round trip
// overlaps the item's work; near the end (and in batches of about one wave)
// it takes it when the item ends, so that no worker holds an item that an
// idle one could run.
constexpr unsigned int kNoTicket = 0xffffffffu;

__device__ __forceinline__ unsigned int early_ticket(bool leader, unsigned int *ctl, int phase,
                                                     unsigned int it, uint64_t total,
                                                     uint64_t workers)
{
    return leader && it + workers < total ? atomicAdd(ctl + kCtlTicket0 + phase, 1u) : kNoTicket;
}

__device__ __forceinline__ unsigned int late_ticket(bool leader, unsigned int *ctl, int phase,
                                                    unsigned int nxt)
{
    return leader && nxt == kNoTicket ? atomicAdd(ctl + kCtlTicket0 + phase, 1u) : nxt;
}

// The barrier of one half: named barrier 1 or 2 over its kHalf threads
// (immediate ids, so the kernel reserves three barriers, not all sixteen).
struct HalfSync {
    int half;
    __device__ __forceinline__ void operator()() const
    {
        static_assert(kHalf == 128, "the barrier counts below are kHalf");
        if (half)
            asm volatile("bar.sync 2, 128;" ::: "memory");
        else
            asm volatile("bar.sync 1, 128;" ::: "memory");
    }
};

// Thread 0 of the half's value of t, for every thread of the half (a
// barrier of the half first, so it also ends the half's work before).
__device__ __forceinline__ unsigned int half_broadcast(unsigned int t, HalfSync hs)
{
    __shared__ unsigned int s_h[2];
    hs();
    if ((threadIdx.x & (kHalf - 1)) == 0)
        s_h[hs.half] = t;
    hs();
    return s_h[hs.half];
}

// ------------------------------------------------------------------ compress
__global__ void __launch_bounds__(kBatchBlock, 2) k_batch_compress(BatchArgs a)
{
    extern __shared__ uint4 smem_raw[];
    __shared__ unsigned long long s_hist[256];
    __shared__ uint32_t s_len[256];
    __shared__ uint32_t s_bits[kBatchBlock];
    __shared__ unsigned long long s_scan[kBatchWarps];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t total_units = a.unit_base[a.count];

    // phase 0: clear the per-buffer statuses; record the owner of every unit
    // and encode item (one search each, all at once), so that the phases
    // below find a unit's or an item's buffer with one load
    for (uint32_t b = blockIdx.x * kBatchBlock + tid; b < a.count; b += gridDim.x * kBatchBlock)
        *a.bufs[b].status = 0;
    const uint64_t total_items = a.item_base[a.count];
    {
        const uint64_t t0 = (uint64_t)blockIdx.x * kBatchBlock + tid, nt = (uint64_t)gridDim.x * kBatchBlock;
        for (uint64_t g = t0; g < total_units; g += nt) {
            const uint32_t b = find_owner(a.unit_base, a.count, g);
            const uint64_t at = (g - a.unit_base[b]) * kUnitSymbols, n = a.bufs[b].in_bytes;
            const uintptr_t p = reinterpret_cast<uintptr_t>(a.bufs[b].in + at);
            a.unit_owner[g] = make_uint4((uint32_t)p, (uint32_t)((uint64_t)p >> 32),
                                         (uint32_t)(n - at < kUnitSymbols ? n - at : kUnitSymbols), b);
        }
        for (uint64_t it = t0; it < total_items; it += nt) {
            const uint32_t b = find_owner(a.item_base, a.count, it);
            const uint64_t u0 = a.unit_base[b];
            a.item_owner[it] = make_uint4(b, (uint32_t)(it - a.item_base[b]), (uint32_t)u0,
                                          (uint32_t)(u0 >> 32));
        }
    }
    if (!grid_barrier(a.ctl, a.fail, a.barrier_extra)) {
        fail_all(a.bufs, a.count);
        return;
    }

    // phase 1: per-unit histograms (columns never cleared: folds are
    // differenced).  Two sets of columns, used by alternate units: a unit's
    // counts go to one set while the other set's fold of the unit before may
    // still run, so one CTA barrier per unit suffices (the next unit counted
    // into a set starts after the barrier that follows the fold of that set)
    {
        uint32_t *cnt = reinterpret_cast<uint32_t *>(smem_raw);  // [2][256][32]
        for (int i = tid; i < 2 * 256 * 32; i += kBatchBlock)
            cnt[i] = 0;
        const uint32_t col0 = smem_u32(cnt) + 4u * lane;
        uint32_t prev0 = 0u, prev1 = 0u;  // folds of each set at its previous unit
        uint32_t set = 0;
        uint4 v[hst::kVecPerThread];
        // a unit is counted while the next one's bytes and the owner entry of
        // the one after are in flight
        const uint64_t G = gridDim.x;
        uint64_t g = blockIdx.x;
        const uint4 none = make_uint4(0u, 0u, 0u, 0u);
        uint4 o0 = g < total_units ? a.unit_owner[g] : none;
        uint4 o1 = g + G < total_units ? a.unit_owner[g + G] : none;
        if (g < total_units)
            hst::load_unit(unit_ptr(o0), o0.z, 0, v);
        __syncthreads();
        for (; g < total_units; g += G) {
            uint4 cur[hst::kVecPerThread];
#pragma unroll
            for (int j = 0; j < hst::kVecPerThread; ++j)
                cur[j] = v[j];
            const uint4 co = o0;
            const uint64_t gn = g + G;
            if (gn < total_units)
                hst::load_unit(unit_ptr(o1), o1.z, 0, v);
            o0 = o1;
            if (gn + G < total_units)
                o1 = a.unit_owner[gn + G];
            hst::count_unit(unit_ptr(co), co.z, 0, cur, col0 + set * (256 * 32 * 4));
            __syncthreads();
            const uint32_t s = hst::fold_bin(cnt + set * (256 * 32), tid);
            a.unit_hist[g * 256 + tid] = (uint16_t)(s - (set ? prev1 : prev0));
            if (set)
                prev1 = s;
            else
                prev0 = s;
            set ^= 1u;
        }
    }
    if (!grid_barrier(a.ctl, a.fail, a.barrier_extra)) {
        fail_all(a.bufs, a.count);
        return;
    }

    // phase 2: per buffer codebook, unit offsets and header
    {
        cbk::CodebookShared &csh = *reinterpret_cast<cbk::CodebookShared *>(smem_raw);
        for (unsigned int b = take_ticket(a.ctl, 0); b < a.count;) {
            const unsigned int nxt = early_ticket(tid == 0, a.ctl, 0, b, a.count, gridDim.x);
            const BatchBuf B = a.bufs[b];
            const uint64_t u0 = a.unit_base[b], nu = a.unit_base[b + 1] - u0;
            unsigned long long h = 0;
            for (uint64_t u = 0; u < nu; ++u)
                h += a.unit_hist[(u0 + u) * 256 + tid];
            s_hist[tid] = h;
            __syncthreads();
            cbk::build_codebook(s_hist, a.cbs + b, B.status, csh);
            __syncthreads();
            s_len[tid] = a.cbs[b].len[tid];
            __syncthreads();
            unsigned long long *off = a.unit_off + u0 + b;
            // unit bit counts, 256 units at a time: unit i of a tile goes to
            // warp i mod 8 (one coalesced 512-byte row: lane l dots bins
            // 8l..8l+7 with their code lengths, the warp sums), through
            // shared memory to thread i, and the tile is scanned with a
            // running carry
            uint32_t L8[8];
#pragma unroll
            for (int j = 0; j < 8; ++j)
                L8[j] = s_len[8 * lane + j];
            unsigned long long carry = 0;
            for (uint64_t t0 = 0; t0 < nu; t0 += kBatchBlock) {
                const uint64_t u = t0 + tid;
#pragma unroll 4
                for (int k = 0; k < kBatchBlock / kBatchWarps; ++k) {
                    const uint32_t i = (uint32_t)k * kBatchWarps + (uint32_t)warp;
                    if (t0 + i < nu) {  // warp-uniform
                        const uint4 q = __ldcg(reinterpret_cast<const uint4 *>(
                                                   a.unit_hist + (u0 + t0 + i) * 256) + lane);
                        const uint32_t d = (q.x & 0xffffu) * L8[0] + (q.x >> 16) * L8[1] +
                                           (q.y & 0xffffu) * L8[2] + (q.y >> 16) * L8[3] +
                                           (q.z & 0xffffu) * L8[4] + (q.z >> 16) * L8[5] +
                                           (q.w & 0xffffu) * L8[6] + (q.w >> 16) * L8[7];
                        const uint32_t t = __reduce_add_sync(0xffffffffu, d);
                        if (lane == 0)
                            s_bits[i] = t;
                    }
                }
                __syncthreads();
                const uint32_t bits = u < nu ? s_bits[tid] : 0u;
                unsigned long long x = bits;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const unsigned long long y = __shfl_up_sync(0xffffffffu, x, d);
                    if (lane >= d)
                        x += y;
                }
                if (lane == 31)
                    s_scan[warp] = x;
                __syncthreads();
                unsigned long long before = 0, tot = 0;
                for (int w = 0; w < kBatchWarps; ++w) {
                    if (w < warp)
                        before += s_scan[w];
                    tot += s_scan[w];
                }
                if (u < nu)
                    off[u] = carry + before + x - bits;
                carry += tot;
                __syncthreads();
            }
            if (tid == 0)
                off[nu] = carry;
            __syncthreads();
            const enc::Job J = enc::make_job(B.in, B.in_bytes, a.cs, off, B.out, B.out_cap);
            if (!uniform_failed(B.status))
                enc::write_header(J, a.cbs + b, B.out_bytes, B.status);
            b = cta_broadcast(late_ticket(tid == 0, a.ctl, 0, nxt));
        }
    }
    if (!grid_barrier(a.ctl, a.fail, a.barrier_extra)) {
        fail_all(a.bufs, a.count);
        return;
    }

    // phase 3: encode, each half of the CTA on its own items with its own
    // code table (its named barrier; no CTA barrier from here on)
    {
        const int half = warp / kHalfWarps, htid = tid & (kHalf - 1), hwarp = warp % kHalfWarps;
        const HalfSync hs{half};
        uint32_t *tbl = reinterpret_cast<uint32_t *>(smem_raw) + half * enc::kTblWords;
        uint32_t *wob = reinterpret_cast<uint32_t *>(smem_raw) + 2 * enc::kTblWords + warp * enc::kWarpObuf;
        uint32_t have = 0xffffffffu;  // buffer whose table is loaded
        bool fast = true;
        int group = 1;
        const unsigned int t0 = htid == 0 ? atomicAdd(a.ctl + kCtlTicket0 + 1, 1u) : 0u;
        for (unsigned int it = half_broadcast(t0, hs); it < total_items;) {
            const unsigned int nxt =
                early_ticket(htid == 0, a.ctl, 1, it, total_items, 2ull * gridDim.x);
            const uint4 ow = a.item_owner[it];  // (buffer, item within it, first unit)
            const uint32_t b = ow.x;
            const BatchBuf B = a.bufs[b];
            const bool failed =  // this buffer's codebook failed
                half_broadcast(htid == 0 ? (unsigned int)chain_failed(B.status) : 0u, hs) != 0;
            if (!failed) {
                if (b != have) {
                    const uint32_t max_len = a.cbs[b].max_len;
                    fast = max_len <= (uint32_t)enc::kFastMaxLen;
                    group = enc::emit_group(max_len);
                    enc::build_table(a.cbs + b, tbl, fast, htid, kHalf);
                    hs();
                    have = b;
                }
                const uint64_t u0 = ow.z | ((uint64_t)ow.w << 32);
                const enc::Job J =
                    enc::make_job(B.in, B.in_bytes, a.cs, a.unit_off + u0 + b, B.out, B.out_cap);
                const uint64_t u = (uint64_t)ow.y * kUnitsPerItem + hwarp;
                bool overflow = false;
                if (u < J.units)
                    overflow = enc::encode_unit(J, u, tbl, fast, group, wob);
                if (overflow)
                    set_status(B.status, HUFF_ERR_CAPACITY);
            }
            // also: the table may be rebuilt for the next item
            it = half_broadcast(late_ticket(htid == 0, a.ctl, 1, nxt), hs);
        }
    }
}

// ------------------------------------------------------------------ decompress
// Each half of a CTA (4 warps, its own named barrier) decodes items of its
// own buffer: an item is one task per warp of the half, so a small buffer
// leaves fewer lanes idle than with items of the whole CTA.  One copy of the
// lookup tables per half (tables are rebuilt per buffer, and most buffers of
// a batch are small); dynamic shared memory as in decode.cu: the two halves'
// tables, then from the next 4 KiB boundary a 4 KiB output block per warp,
// then a 4 KiB input block per warp (a half builds its tables with its own
// warps' input blocks as scratch).
constexpr int kBatchCopies = 1;
constexpr size_t kDecompTables = (sizeof(dec::DecodeShared<kBatchCopies>) + 15) & ~size_t(15);
constexpr size_t kDecompressSmem = 2 * kDecompTables + 4096 + (size_t)kBatchWarps * 2 * 4096;

__global__ void __launch_bounds__(kBatchBlock, 2) k_batch_decompress(BatchArgs a)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    const uint32_t rings = (smem_u32(dsm) + 2u * (uint32_t)kDecompTables + 4095u) & ~4095u;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // phase 1: statuses and work sizes from the headers
    for (uint32_t b = blockIdx.x * kBatchBlock + tid; b < a.count; b += gridDim.x * kBatchBlock) {
        const BatchBuf B = a.bufs[b];
        *B.status = 0;
        uint64_t items = 1;  // a malformed header still gets one item to report it
        if (B.in_bytes >= kHeaderBytes) {
            const uint64_t n = *reinterpret_cast<const uint64_t *>(B.in + 256);
            const uint32_t cs = *reinterpret_cast<const uint32_t *>(B.in + 264);
            if (chunk_symbols_valid(cs)) {
                const uint64_t chunks = n / cs + (n % cs != 0);
                if (chunks <= (B.in_bytes - kHeaderBytes) / 8) {
                    const uint32_t S = dec::pick_split(chunks, a.min_lanes);
                    const uint64_t tasks = (chunks + (32 / S) - 1) / (32 / S);
                    items = tasks ? (tasks + kTasksPerItem - 1) / kTasksPerItem : 1;
                }
            }
        }
        a.dec_items[b] = items;
    }
    if (!grid_barrier(a.ctl, a.fail, a.barrier_extra)) {
        fail_all(a.bufs, a.count);
        return;
    }
    // phase 2: exclusive scan of the work sizes (CTA 0), in place
    if (blockIdx.x == 0) {
        __shared__ unsigned long long s_part[kBatchBlock];
        const uint32_t per = (a.count + kBatchBlock - 1) / kBatchBlock;
        const uint32_t b0 = tid * per, b1 = min(a.count, b0 + per);
        unsigned long long own = 0;
        for (uint32_t b = b0; b < b1; ++b)
            own += a.dec_items[b];
        s_part[tid] = own;
        __syncthreads();
        unsigned long long before = 0;
        for (int t = 0; t < tid; ++t)
            before += s_part[t];
        for (uint32_t b = b0; b < b1; ++b) {
            const unsigned long long v = a.dec_items[b];
            a.dec_items[b] = before;
            before += v;
        }
        if (tid == kBatchBlock - 1)
            a.dec_items[a.count] = before;
    }
    if (!grid_barrier(a.ctl, a.fail, a.barrier_extra)) {
        fail_all(a.bufs, a.count);
        return;
    }

    // phase 3: decode items, each half of the CTA on its own (its named
    // barrier; no CTA barrier from here on)
    const int half = warp / kHalfWarps, htid = tid & (kHalf - 1), hwarp = warp % kHalfWarps;
    const HalfSync hs{half};
    dec::DecodeShared<kBatchCopies> &sh =
        *reinterpret_cast<dec::DecodeShared<kBatchCopies> *>(dsm + half * kDecompTables);
    uint16_t *scratch = reinterpret_cast<uint16_t *>(
        dsm + (rings - smem_u32(dsm)) + (kBatchWarps + half * kHalfWarps) * 4096);
    const uint32_t out_s = rings + warp * 4096 + lane * 4;
    const uint32_t in_s = rings + (kBatchWarps + warp) * 4096 + lane * 16;
    const uint64_t total_items = a.dec_items[a.count];
    uint32_t have = 0xffffffffu;
    bool ready = false;
    dec::StreamInfo si;
    uint32_t S = 1;
    const unsigned int t0 = htid == 0 ? atomicAdd(a.ctl + kCtlTicket0 + 2, 1u) : 0u;
    for (unsigned int it = half_broadcast(t0, hs); it < total_items;) {
        const unsigned int nxt =
            early_ticket(htid == 0, a.ctl, 2, it, total_items, 2ull * gridDim.x);
        const uint32_t b = find_owner(a.dec_items, a.count, it);
        const BatchBuf B = a.bufs[b];
        if (b != have) {
            ready = dec::prepare<kHalf>(B.in, B.in_bytes, B.out, B.out_cap, B.out_bytes, B.status,
                                        it == a.dec_items[b] && htid == 0, sh, scratch, si, htid,
                                        hs);
            if (ready)
                S = dec::pick_split(si.chunks, a.min_lanes);
            have = b;
        }
        const bool failed =
            half_broadcast(htid == 0 ? (unsigned int)chain_failed(B.status) : 0u, hs) != 0;
        if (ready && !failed) {
            const uint64_t tasks = (si.chunks + (32 / S) - 1) / (32 / S);
            const uint64_t task = (uint64_t)(it - a.dec_items[b]) * kTasksPerItem + hwarp;
            if (task < tasks && dec::decode_task(si, S, task, in_s, out_s)) {
                if (lane == 0)
                    set_status(B.status, HUFF_ERR_CORRUPT_STREAM);
            }
        }
        // also: the tables may be rebuilt for the next item
        it = half_broadcast(late_ticket(htid == 0, a.ctl, 2, nxt), hs);
    }
}

// phase 1's two sets of histogram columns, or phase 3's two code tables and
// word buffers, whichever is larger
constexpr int kCompressSmem = (2 * enc::kTblWords + kBatchWarps * enc::kWarpObuf) * 4 > 2 * 256 * 32 * 4
                                  ? (2 * enc::kTblWords + kBatchWarps * enc::kWarpObuf) * 4
                                  : 2 * 256 * 32 * 4;

}  // namespace

}  // namespace huff

// ====================================================================== host
namespace huff {

// Device block of one batch: control words, descriptors, prefix arrays and
// (compress) per-unit histograms, unit offsets, codebooks and the owners of
// units and encode items.
void batch_layout(const huff_batch_desc_t *descs, uint32_t count, huff_op_t op, BatchLayout &L)
{
    auto al = [](uint64_t x) { return (x + 255) & ~uint64_t(255); };
    L.count = count;
    L.op = op;
    L.bufs.resize(count);
    L.unit_base.assign(count + 1, 0);
    L.item_base.assign(count + 1, 0);
    for (uint32_t i = 0; i < count; ++i) {
        L.bufs[i] = {descs[i].d_in, descs[i].in_bytes, descs[i].d_out, descs[i].out_cap,
                     reinterpret_cast<unsigned long long *>(descs[i].d_out_bytes),
                     descs[i].d_status};
        const uint64_t units = op == HUFF_BATCH_COMPRESS
                                   ? (descs[i].in_bytes + kUnitSymbols - 1) / kUnitSymbols
                                   : 0;
        L.unit_base[i + 1] = L.unit_base[i] + units;
        L.item_base[i + 1] = L.item_base[i] + (units + kUnitsPerItem - 1) / kUnitsPerItem;
    }
    const uint64_t total_units = L.unit_base[count];
    uint64_t off = 0;
    L.o_ctl = off;
    off = al(off + sizeof(unsigned int) * kCtlWords + sizeof(int32_t));
    L.o_bufs = off;
    off = al(off + sizeof(BatchBuf) * count);
    L.o_ub = off;
    off = al(off + 8 * (count + 1));
    L.o_ib = off;
    off = al(off + 8 * (count + 1));
    L.o_di = off;
    off = al(off + 8 * (count + 1));
    L.o_uh = L.o_uo = L.o_cb = L.o_uw = L.o_iw = off;
    if (op == HUFF_BATCH_COMPRESS) {
        L.o_uh = off;
        off = al(off + 512 * total_units);
        L.o_uo = off;
        off = al(off + 8 * (total_units + count));
        L.o_cb = off;
        off = al(off + sizeof(huff_codebook_t) * count);
        L.o_uw = off;
        off = al(off + 16 * total_units);
        L.o_iw = off;
        off = al(off + 16 * L.item_base[count]);
    }
    L.bytes = off;
    // the host-side part copied to the device: descriptors and prefixes
    L.upload_bytes = L.o_di;
}

BatchArgs batch_args(const BatchLayout &L, void *d_block, uint32_t cs, uint32_t lanes,
                     uint32_t barrier_extra)
{
    uint8_t *blk = static_cast<uint8_t *>(d_block);
    BatchArgs a;
    a.bufs = reinterpret_cast<const BatchBuf *>(blk + L.o_bufs);
    a.count = L.count;
    a.cs = cs;
    a.unit_base = reinterpret_cast<const uint64_t *>(blk + L.o_ub);
    a.item_base = reinterpret_cast<const uint64_t *>(blk + L.o_ib);
    a.dec_items = reinterpret_cast<uint64_t *>(blk + L.o_di);
    const bool c = L.op == HUFF_BATCH_COMPRESS;
    a.unit_hist = c ? reinterpret_cast<uint16_t *>(blk + L.o_uh) : nullptr;
    a.unit_off = c ? reinterpret_cast<unsigned long long *>(blk + L.o_uo) : nullptr;
    a.cbs = c ? reinterpret_cast<huff_codebook_t *>(blk + L.o_cb) : nullptr;
    a.unit_owner = c ? reinterpret_cast<uint4 *>(blk + L.o_uw) : nullptr;
    a.item_owner = c ? reinterpret_cast<uint4 *>(blk + L.o_iw) : nullptr;
    a.min_lanes = lanes;
    a.ctl = reinterpret_cast<unsigned int *>(blk + L.o_ctl);
    a.fail = reinterpret_cast<int32_t *>(blk + L.o_ctl + sizeof(unsigned int) * kCtlWords);
    a.barrier_extra = barrier_extra;
    return a;
}

// Fill `host` (upload_bytes, ideally pinned) with the descriptors and prefixes
// and copy it to the start of the device block.
cudaError_t batch_upload(const BatchLayout &L, void *d_block, uint8_t *host, cudaStream_t s)
{
    std::memset(host, 0, L.upload_bytes);
    std::memcpy(host + L.o_bufs, L.bufs.data(), sizeof(BatchBuf) * L.count);
    std::memcpy(host + L.o_ub, L.unit_base.data(), 8 * (L.count + 1));
    std::memcpy(host + L.o_ib, L.item_base.data(), 8 * (L.count + 1));
    return cudaMemcpyAsync(d_block, host, L.upload_bytes, cudaMemcpyHostToDevice, s);
}

KernelSetup g_compress_setup, g_decompress_setup;

// Resident CTAs per SM of the batch kernel for `op` on the current device
// (0 on error).
int batch_occupancy(huff_op_t op)
{
    int per_sm = 0;
    const cudaError_t err =
        op == HUFF_BATCH_COMPRESS
            ? kernel_setup(g_compress_setup, (const void *)k_batch_compress, kBatchBlock,
                           kCompressSmem, &per_sm)
            : kernel_setup(g_decompress_setup, (const void *)k_batch_decompress, kBatchBlock,
                           kDecompressSmem, &per_sm);
    return err == cudaSuccess ? per_sm : 0;
}

// Clear the control words and launch the cooperative batch kernel.
cudaError_t batch_launch(huff_op_t op, const BatchArgs &args, unsigned grid, cudaStream_t s)
{
    cudaError_t err = cudaMemsetAsync(args.ctl, 0, sizeof(unsigned int) * kCtlWords + sizeof(int32_t), s);
    if (err != cudaSuccess)
        return err;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kBatchBlock);
    cfg.dynamicSmemBytes = op == HUFF_BATCH_COMPRESS ? kCompressSmem : kDecompressSmem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return op == HUFF_BATCH_COMPRESS ? cudaLaunchKernelEx(&cfg, k_batch_compress, args)
                                     : cudaLaunchKernelEx(&cfg, k_batch_decompress, args);
}

// Argument checks shared by plans and served rounds.
huff_status_t batch_check(const huff_batch_desc_t *descs, uint32_t count, huff_op_t op,
                          const huff_batch_params_t &prm)
{
    if (!descs || count == 0 || (op != HUFF_BATCH_COMPRESS && op != HUFF_BATCH_DECOMPRESS))
        return HUFF_ERR_INVALID_ARG;
    if (op == HUFF_BATCH_COMPRESS && !chunk_symbols_valid(prm.chunk_symbols))
        return HUFF_ERR_INVALID_ARG;
    if (prm.decode_lanes == 0 || prm.decode_lanes > 65536 || prm.barrier_extra > 65536)
        return HUFF_ERR_INVALID_ARG;
    for (uint32_t i = 0; i < count; ++i) {
        const huff_batch_desc_t &d = descs[i];
        if (!d.d_out || !d.d_out_bytes || !d.d_status || (d.in_bytes && !d.d_in) ||
            (reinterpret_cast<uintptr_t>(d.d_in) & 15) ||
            (reinterpret_cast<uintptr_t>(d.d_out) & 15))
            return HUFF_ERR_INVALID_ARG;
        if (op == HUFF_BATCH_COMPRESS &&
            (d.in_bytes > (uint64_t)UINT32_MAX * kUnitSymbols ||
             d.out_cap < kHeaderBytes + 8 * ceil_div_u64(d.in_bytes, prm.chunk_symbols)))
            return HUFF_ERR_INVALID_ARG;
    }
    return HUFF_OK;
}

}  // namespace huff

using namespace huff;

struct huff_batch_plan {
    huff_op_t op;
    huff_batch_params_t params;
    uint32_t count;
    unsigned grid;
    void *d_block;  // device memory owned by the plan
    BatchArgs args;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

namespace {

void free_plan(huff_batch_plan_t *p)
{
    if (!p)
        return;
    if (p->exec)
        cudaGraphExecDestroy(p->exec);
    if (p->graph)
        cudaGraphDestroy(p->graph);
    if (p->d_block)
        cudaFree(p->d_block);
    delete p;
}

}  // namespace

extern "C" {

void huff_batch_default_params(huff_batch_params_t *params)
{
    if (!params)
        return;
    params->chunk_symbols = HUFF_DEFAULT_CHUNK_SYMBOLS;
    params->ctas_per_sm = 0;  // as many as fit
    params->decode_lanes = 128;
    params->use_graph = 1;
    params->barrier_extra = 0;
}

huff_status_t huff_batch_plan(const huff_batch_desc_t *descs, uint32_t count, huff_op_t op,
                              const huff_batch_params_t *params, huff_batch_plan_t **out_plan)
{
    HUFF_API_RANGE("huff_batch_plan");
    if (!out_plan)
        return HUFF_ERR_INVALID_ARG;
    *out_plan = nullptr;
    huff_batch_params_t prm;
    huff_batch_default_params(&prm);
    if (params)
        prm = *params;
    huff_status_t st = batch_check(descs, count, op, prm);
    if (st != HUFF_OK)
        return st;

    huff_batch_plan_t *p = new (std::nothrow) huff_batch_plan_t();
    if (!p)
        return HUFF_ERR_CUDA;
    std::memset(p, 0, sizeof(*p));
    p->op = op;
    p->params = prm;
    p->count = count;
    BatchLayout L;
    batch_layout(descs, count, op, L);
    if (cudaMalloc(&p->d_block, L.bytes) != cudaSuccess) {
        free_plan(p);
        return HUFF_ERR_CUDA;
    }
    // upload on a private stream: the legacy default stream would wait for
    // (and hold up) every other blocking stream of the process
    cudaStream_t up;
    if (cudaStreamCreateWithFlags(&up, cudaStreamNonBlocking) != cudaSuccess) {
        free_plan(p);
        return HUFF_ERR_CUDA;
    }
    std::vector<uint8_t> host(L.upload_bytes);
    const bool uploaded = batch_upload(L, p->d_block, host.data(), up) == cudaSuccess &&
                          cudaStreamSynchronize(up) == cudaSuccess;
    cudaStreamDestroy(up);
    if (!uploaded) {
        free_plan(p);
        return HUFF_ERR_CUDA;
    }
    p->args = batch_args(L, p->d_block, prm.chunk_symbols, prm.decode_lanes, prm.barrier_extra);
    int per_sm = batch_occupancy(op);
    if (per_sm < 1) {
        free_plan(p);
        return HUFF_ERR_CUDA;
    }
    if (prm.ctas_per_sm && (int)prm.ctas_per_sm < per_sm)
        per_sm = (int)prm.ctas_per_sm;
    p->grid = (unsigned)(device_sm_count() * per_sm);

    if (prm.use_graph) {
        cudaStream_t cs;
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
            free_plan(p);
            return HUFF_ERR_CUDA;
        }
        bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            const cudaError_t le = batch_launch(op, p->args, p->grid, cs);
            ok = cudaStreamEndCapture(cs, &p->graph) == cudaSuccess && le == cudaSuccess;
        }
        if (ok)
            ok = cudaGraphInstantiate(&p->exec, p->graph, 0) == cudaSuccess;
        cudaStreamDestroy(cs);
        if (!ok) {  // fall back to direct launches
            cudaGetLastError();
            if (p->exec)
                cudaGraphExecDestroy(p->exec);
            if (p->graph)
                cudaGraphDestroy(p->graph);
            p->exec = nullptr;
            p->graph = nullptr;
            p->params.use_graph = 0;
        }
    }
    *out_plan = p;
    return HUFF_OK;
}

huff_status_t huff_batch_run(huff_batch_plan_t *plan, huff_stream_t stream)
{
    HUFF_API_RANGE("huff_batch_run");
    if (!plan)
        return HUFF_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (plan->exec)
        return cudaGraphLaunch(plan->exec, s) == cudaSuccess ? HUFF_OK : HUFF_ERR_CUDA;
    return batch_launch(plan->op, plan->args, plan->grid, s) == cudaSuccess ? HUFF_OK
                                                                              : HUFF_ERR_CUDA;
}

huff_status_t huff_batch_info(const huff_batch_plan_t *plan, huff_batch_params_t *params,
                              uint32_t *grid, int32_t *used_graph)
{
    if (!plan)
        return HUFF_ERR_INVALID_ARG;
    if (params)
        *params = plan->params;
    if (grid)
        *grid = plan->grid;
    if (used_graph)
        *used_graph = plan->exec != nullptr;
    return HUFF_OK;
}

void huff_batch_destroy(huff_batch_plan_t *plan) { free_plan(plan); }

}  // extern "C"
