// Decoder device routines, shared by the single-stream kernel (decode.cu)
// and the batched kernel (batch.cu).  See decode.cu for the design.
#pragma once

#include "huff_internal.cuh"

namespace huff {
namespace dec {

constexpr int kLutBits = 12;
constexpr int kLutSize = 1 << kLutBits;
constexpr int kInRing = 32;   // input ring: words per lane
constexpr int kOutRing = 8;   // output ring: 32 bytes per lane
constexpr int kWindow = 8;    // lookups between ring maintenance


struct Tables {
    const uint32_t *lut;
    const uint32_t *count;
    const uint32_t *first;
    const uint32_t *start;
    const uint8_t *sorted;
    uint32_t max_len;
};

// Shared-memory state of one stream's decode tables.
struct DecodeShared {
    uint32_t lut[kLutSize];
    uint8_t len_s[256];
    uint8_t sorted[256];
    uint32_t count[kMaxCodeLen + 1];
    uint32_t first[kMaxCodeLen + 1];
    uint32_t start[kMaxCodeLen + 1];
    unsigned long long s_kraft;
    int s_max, s_nsym, s_bad;
};

// What a warp needs to decode chunks of one stream.
struct StreamInfo {
    const uint8_t *stream;
    uint8_t *out;
    uint64_t n;
    uint32_t cs;
    uint64_t chunks;
    uint64_t pay_words;
    uint64_t pbits;
    const uint64_t *offs;
    const uint8_t *pay;
    Tables T;
};

// Codes longer than the table: canonical search by length on a 32-bit window.
__device__ __forceinline__ bool long_code(const Tables &T, uint64_t buf, uint32_t &L, uint32_t &sym)
{
    const uint32_t v = (uint32_t)(buf >> 32);
    for (uint32_t l = kLutBits + 1; l <= T.max_len; ++l) {
        const uint32_t cv = v >> (32 - l);
        if (T.count[l] && cv - T.first[l] < T.count[l]) {
            L = l;
            sym = T.sorted[T.start[l] + cv - T.first[l]];
            return true;
        }
    }
    return false;
}

// Bit reader over the payload's u32 words.  Words come in blocks of four
// (two 8-byte loads); the block after the current one is always in flight,
// so a register is never read right after its load was issued, and an L2
// prefetch runs 256 bytes ahead.  Words past the payload read as zero.
struct Reader {
    const uint2 *pairs;
    uint64_t nwords;
    uint64_t next_blk;
    uint2 c0, c1, n0, n1;
    uint32_t idx;  // next word of the current block
    uint64_t buf;  // valid bits left-aligned
    int have;

    __device__ __forceinline__ void load_block(uint64_t b, uint2 &x0, uint2 &x1) const
    {
        const uint64_t w = 4 * b;
        if (w + 4 <= nwords) {
            x0 = pairs[2 * b];
            x1 = pairs[2 * b + 1];
        } else {
            const uint32_t *words = reinterpret_cast<const uint32_t *>(pairs);
            x0.x = w < nwords ? words[w] : 0u;
            x0.y = w + 1 < nwords ? words[w + 1] : 0u;
            x1.x = w + 2 < nwords ? words[w + 2] : 0u;
            x1.y = 0u;
        }
    }
    __device__ __forceinline__ uint32_t next_word()
    {
        const uint32_t w = idx == 0 ? c0.x : idx == 1 ? c0.y : idx == 2 ? c1.x : c1.y;
        if (++idx == 4) {
            idx = 0;
            c0 = n0;
            c1 = n1;
            load_block(next_blk, n0, n1);
            ++next_blk;
            if ((next_blk & 7) == 0 && 4 * (next_blk + 16) < nwords)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(pairs + 2 * (next_blk + 16)));
        }
        return w;
    }
    __device__ __forceinline__ void init(const uint8_t *pay, uint64_t nw, uint64_t pos)
    {
        pairs = reinterpret_cast<const uint2 *>(pay);
        nwords = nw;
        const uint64_t wi = pos >> 5, b = wi >> 2;
        load_block(b, c0, c1);
        load_block(b + 1, n0, n1);
        next_blk = b + 2;
        idx = (uint32_t)(wi & 3);
        buf = ((uint64_t)next_word() << 32) << (pos & 31);
        have = 32 - (int)(pos & 31);
    }
    __device__ __forceinline__ void refill()
    {
        if (have <= 32) {
            buf |= (uint64_t)next_word() << (32 - have);
            have += 32;
        }
    }
    __device__ __forceinline__ void consume(uint32_t L)
    {
        buf <<= L;
        have -= (int)L;
    }
};

__device__ __forceinline__ void cp_async4(uint32_t *dst, const uint32_t *src, bool valid)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src),
                 "r"(valid ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Bit stream of one lane fed through its column of the warp's input ring
// (word slot w of lane l at ring[w * 32 + l]).  Word indices are relative to
// w0, the payload word that holds the chunk's first bit.  Invariants: after
// every top-up at least 25 words are requested beyond the next one to read,
// groups are 4 words, and the two most recent groups may still be in flight,
// so the >= 9 words a window can touch have landed.
struct RingStream {
    uint32_t *col;          // this lane's column
    const uint32_t *words;  // payload
    uint64_t nwords;
    uint64_t w0;
    uint32_t widx;    // next word to move into the bit buffer
    uint32_t fidx;    // next word to request
    uint32_t nxt;     // word widx, preloaded
    uint32_t bh, bl;  // bit buffer, valid bits left-aligned in bh:bl
    int have;

    __device__ __forceinline__ void fetch4()
    {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint64_t aw = w0 + fidx + j;
            const bool ok = aw < nwords;
            cp_async4(col + ((fidx + j) & (kInRing - 1)) * 32, words + (ok ? aw : 0), ok);
        }
        fidx += 4;
        cp_async_commit();
    }
    __device__ __forceinline__ void top_up()
    {
        if (fidx - widx <= kInRing - 8)
            fetch4();
        if (fidx - widx <= kInRing - 8)
            fetch4();
    }
    // start at bit `pbit` counted from the first bit of word w0
    __device__ __forceinline__ void init(uint32_t *column, const uint32_t *pay, uint64_t nw,
                                         uint64_t word0, uint32_t pbit)
    {
        col = column;
        words = pay;
        nwords = nw;
        w0 = word0;
        widx = pbit >> 5;
        fidx = widx;
#pragma unroll
        for (int r = 0; r < kInRing / 4; ++r)
            fetch4();
        cp_async_wait<0>();
        const uint32_t sh = pbit & 31;
        bh = col[(widx & (kInRing - 1)) * 32] << sh;
        bl = 0;
        have = 32 - (int)sh;
        ++widx;
        nxt = col[(widx & (kInRing - 1)) * 32];
    }
    // top the buffer up to more than 32 valid bits
    __device__ __forceinline__ void refill()
    {
        if (have <= 32) {
            bh |= __funnelshift_rc(nxt, 0u, (uint32_t)have);  // nxt >> have (0 at 32)
            bl |= nxt << (32 - have);
            have += 32;
            ++widx;
            nxt = col[(widx & (kInRing - 1)) * 32];
        }
    }
    __device__ __forceinline__ uint32_t peek12() const { return bh >> (32 - kLutBits); }
    __device__ __forceinline__ uint64_t buf64() const { return ((uint64_t)bh << 32) | bl; }
    // drop L < 32 bits
    __device__ __forceinline__ void consume_small(uint32_t L)
    {
        bh = __funnelshift_l(bl, bh, L);
        bl <<= L;
        have -= (int)L;
    }
    // drop L <= 32 bits
    __device__ __forceinline__ void consume(uint32_t L)
    {
        bh = __funnelshift_lc(bl, bh, L);
        bl = L >= 32 ? 0u : bl << L;
        have -= (int)L;
    }
};

// Count codewords from bit `pos` (relative to the chunk's first bit `cbase`)
// until the first boundary at or past `stop`.  Bit i of bmap is set when a
// codeword starts at pos0 + i (i < 64).  Invalid bits (possible off the true
// path) count as 1-bit codewords.
__device__ __forceinline__ void count_codes(const Tables &T, const uint8_t *pay, uint64_t nw,
                                            uint64_t cbase, uint32_t pos, uint32_t stop,
                                            uint32_t &n, uint32_t &e, uint64_t &bmap)
{
    const uint32_t pos0 = pos;
    uint32_t cnt = 0;
    bmap = 1;
    if (pos < stop) {
        Reader rd;
        rd.init(pay, nw, cbase + pos);
        while (pos < stop) {
            rd.refill();
            const uint32_t ent = T.lut[rd.buf >> (64 - kLutBits)];
            uint32_t ns = ent >> 30, L = (ent >> 24) & 31u;
            if (ns == 0) {
                uint32_t sym;
                if (!long_code(T, rd.buf, L, sym))
                    L = 1;
                ns = 1;
            } else if (ns == 2) {
                const uint32_t L0 = (ent >> 16) & 31u;
                if (pos + L0 >= stop) {
                    ns = 1;
                    L = L0;
                } else if (pos + L0 - pos0 < 64) {
                    bmap |= 1ull << (pos + L0 - pos0);
                }
            }
            pos += L;
            if (pos - pos0 < 64)
                bmap |= 1ull << (pos - pos0);
            cnt += ns;
            rd.consume(L);
        }
    }
    n = cnt;
    e = pos;
}

// Sub-segment [g, stop) was counted from g (cnt codewords, exit e, early
// boundaries bmap).  Given its true entry point, walk the true path one
// codeword at a time until it lands on one of the recorded boundaries: from
// there both paths are the same codeword sequence, so only the codewords
// before the meeting point change.  If they do not meet within the recorded
// 64 bits, recount from the entry point.
__device__ __forceinline__ void settle_segment(const Tables &T, const uint8_t *pay, uint64_t nw,
                                               uint64_t cbase, uint32_t g, uint32_t stop,
                                               uint32_t entry, uint64_t bmap, uint32_t cnt1,
                                               uint32_t e1, uint32_t &cnt, uint32_t &e)
{
    uint32_t pos = entry, steps = 0;
    Reader rd;
    bool started = false;
    for (;;) {
        const uint32_t d = pos - g;
        if (d < 64 && ((bmap >> d) & 1)) {  // met: same path from here on
            cnt = steps + cnt1 - __popcll(bmap & ((1ull << d) - 1));
            e = e1;
            return;
        }
        if (pos >= stop) {  // left the sub-segment before meeting
            cnt = steps;
            e = pos;
            return;
        }
        if (d >= 64)
            break;
        if (!started) {
            rd.init(pay, nw, cbase + pos);
            started = true;
        }
        rd.refill();
        const uint32_t ent = T.lut[rd.buf >> (64 - kLutBits)];
        uint32_t L = (ent >> 16) & 31u;  // first code only: every boundary matters
        if ((ent >> 30) == 0) {
            uint32_t sym;
            if (!long_code(T, rd.buf, L, sym))
                L = 1;
        }
        pos += L;
        ++steps;
        rd.consume(L);
    }
    uint64_t unused;
    count_codes(T, pay, nw, cbase, entry, stop, cnt, e, unused);
}

// Validate the stream header and build the decode tables of one stream in
// shared memory (all NT threads of the CTA take part; `reporter` writes *d_n
// and the header errors).  Returns true when there are chunks to decode.
template <int NT>
__device__ __forceinline__ bool prepare(const uint8_t *stream_in, uint64_t bytes, uint8_t *out,
                                        uint64_t cap, unsigned long long *d_n, int32_t *status,
                                        bool reporter, DecodeShared &sh, StreamInfo &si)
{
    const int tid = threadIdx.x;
    const uint8_t *stream = stream_in;
    if (bytes < kHeaderBytes) {
        if (reporter)
            set_status(status, HUFF_ERR_CORRUPT_STREAM);
        return false;
    }
    const uint64_t n = *reinterpret_cast<const uint64_t *>(stream + 256);
    const uint32_t cs = *reinterpret_cast<const uint32_t *>(stream + 264);
    const uint32_t max_field = *reinterpret_cast<const uint32_t *>(stream + 268);
    if (!chunk_symbols_valid(cs)) {
        if (reporter)
            set_status(status, HUFF_ERR_CORRUPT_STREAM);
        return false;
    }
    const uint64_t chunks = n / cs + (n % cs != 0);
    if (chunks > (bytes - kHeaderBytes) / 8) {
        if (reporter)
            set_status(status, HUFF_ERR_CORRUPT_STREAM);
        return false;
    }

    // ---- lengths: range, longest, sh.count, Kraft sum ----
    if (tid <= (int)kMaxCodeLen)
        sh.count[tid] = 0;
    if (tid == 0) {
        sh.s_kraft = 0;
        sh.s_max = 0;
        sh.s_nsym = 0;
        sh.s_bad = 0;
    }
    __syncthreads();
    for (int b = tid; b < 256; b += NT) {
        const uint32_t L = stream[b];
        sh.len_s[b] = (uint8_t)L;
        if (L > kMaxCodeLen) {
            sh.s_bad = 1;
        } else if (L) {
            atomicMax(&sh.s_max, (int)L);
            atomicAdd(&sh.s_nsym, 1);
            atomicAdd(&sh.s_kraft, 1ull << (32 - L));
            atomicAdd(&sh.count[L], 1u);
        }
    }
    __syncthreads();
    const uint32_t max_len = (uint32_t)sh.s_max;
    const int nsym = sh.s_nsym;
    const bool bad_header = sh.s_bad || max_len != max_field || (n > 0 && nsym == 0) ||
                            (nsym == 1 && max_len != 1) ||
                            (nsym >= 2 && sh.s_kraft != (1ull << 32));
    if (bad_header) {
        if (reporter)
            set_status(status, HUFF_ERR_CORRUPT_STREAM);
        return false;
    }
    if (reporter)
        *d_n = n;
    if (n > cap) {
        if (reporter)
            set_status(status, HUFF_ERR_CAPACITY);
        return false;
    }
    if (n == 0)
        return false;

    // ---- canonical tables (RFC 1951 next_code recurrence) ----
    if (tid == 0) {
        uint32_t code = 0, idx = 0;
        for (uint32_t L = 1; L <= kMaxCodeLen; ++L) {
            code = (code + sh.count[L - 1]) << 1;
            sh.first[L] = code;
            sh.start[L] = idx;
            idx += sh.count[L];
        }
    }
    __syncthreads();
    for (int b = tid; b < 256; b += NT) {
        const uint32_t L = sh.len_s[b];
        if (L) {
            uint32_t r = 0;
            for (int j = 0; j < b; ++j)
                r += sh.len_s[j] == L;
            sh.sorted[sh.start[L] + r] = (uint8_t)b;
        }
    }
    __syncthreads();
    // pass 1: the sh.first code of every 12-bit window
    const uint32_t lut_len = max_len < (uint32_t)kLutBits ? max_len : (uint32_t)kLutBits;
    for (int v = tid; v < kLutSize; v += NT) {
        uint32_t ent = 0;
        for (uint32_t L = 1; L <= lut_len; ++L) {
            const uint32_t c = (uint32_t)v >> (kLutBits - L);
            if (sh.count[L] && c - sh.first[L] < sh.count[L]) {
                ent = sh.sorted[sh.start[L] + c - sh.first[L]] | (L << 16) | (L << 24) | (1u << 30);
                break;
            }
        }
        sh.lut[v] = ent;
    }
    __syncthreads();
    // pass 2: append a second code when it fits in the rest of the window
    uint32_t ent2[kLutSize / NT];
#pragma unroll
    for (int i = 0; i < kLutSize / NT; ++i) {
        const int v = tid + i * NT;
        uint32_t ent = sh.lut[v];
        const uint32_t L0 = (ent >> 16) & 31u;
        if (ent && L0 < (uint32_t)kLutBits) {
            const uint32_t nxt = sh.lut[((uint32_t)v << L0) & (kLutSize - 1)];
            const uint32_t L1 = (nxt >> 16) & 31u;
            if (nxt && L0 + L1 <= (uint32_t)kLutBits)
                ent = (ent & 0xffu) | ((nxt & 0xffu) << 8) | (L0 << 16) | ((L0 + L1) << 24) |
                      (2u << 30);
        }
        ent2[i] = ent;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kLutSize / NT; ++i)
        sh.lut[tid + i * NT] = ent2[i];
    __syncthreads();


    const uint64_t pay_words = (bytes - kHeaderBytes - 8 * chunks) / 4;
    const uint64_t pbits = 32 * pay_words;
    const uint64_t *offs = reinterpret_cast<const uint64_t *>(stream + kHeaderBytes);
    const uint8_t *pay = stream + kHeaderBytes + 8 * chunks;

    si.stream = stream;
    si.out = out;
    si.n = n;
    si.cs = cs;
    si.chunks = chunks;
    si.pay_words = pay_words;
    si.pbits = pbits;
    si.offs = offs;
    si.pay = pay;
    si.T.lut = sh.lut;
    si.T.count = sh.count;
    si.T.first = sh.first;
    si.T.start = sh.start;
    si.T.sorted = sh.sorted;
    si.T.max_len = max_len;
    return true;
}

// Sub-segments per chunk: enough decoders for `min_chains` lanes overall.
__device__ __forceinline__ uint32_t pick_split(uint64_t chunks, uint32_t min_chains)
{
    uint32_t S = 1;
    while (S < 32 && chunks * S < min_chains)
        S <<= 1;
    return S;
}

// Decode warp task `task` of stream si with S lanes per chunk (32/S chunks
// per warp).  in_col / out_col: this lane's column of the warp's rings.
// Returns true (warp-uniform) if the stream is corrupt.
__device__ __forceinline__ bool decode_task(const StreamInfo &si, uint32_t S, uint64_t task,
                                        uint32_t *in_col, uint32_t *out_col)
{
    const Tables &T = si.T;
    const uint32_t *lut = T.lut;
    const uint64_t n = si.n, chunks = si.chunks, pbits = si.pbits, pay_words = si.pay_words;
    const uint32_t cs = si.cs;
    const uint64_t *offs = si.offs;
    const uint8_t *pay = si.pay;
    const int lane = threadIdx.x & 31;
    const uint32_t G = 32 / S;
    const uint32_t k = (uint32_t)lane & (S - 1);
    const uint32_t grp = (uint32_t)lane / S;
    uint8_t *out_colb = reinterpret_cast<uint8_t *>(out_col);
    const uint64_t c = task * G + grp;
    const bool valid = c < chunks;
    bool bad = false;
    uint64_t cbase = 0;  // chunk's first bit; positions below are relative to it
    uint32_t lim = 0, m = 0, g = 0, stop = 0;
    if (valid) {
        cbase = offs[c];
        const bool lastc = c + 1 == chunks;
        const uint64_t limit = lastc ? pbits : offs[c + 1];
        m = (uint32_t)(n - c * cs < cs ? n - c * cs : cs);
        // a chunk spans at most 32 bits per symbol; beyond that it is corrupt
        bad = (c == 0 && cbase != 0) || cbase > limit ||
              (!lastc && limit - cbase > 32ull * m);
        if (!bad) {
            const uint64_t span = limit - cbase < 32ull * m ? limit - cbase : 32ull * m;
            lim = (uint32_t)(limit - cbase < 32ull * m ? limit - cbase : 32ull * m + 32);
            g = (uint32_t)(span * k / S);
            stop = (uint32_t)(span * (k + 1) / S);
        }
    }
    const bool work = valid && !bad;

    // 1. count each sub-segment but the last from its cut point
    uint32_t cnt1 = 0, e1 = g;
    uint64_t bmap = 1;
    if (S > 1) {  // uniform: every lane of the warp takes this branch
        RingStream rs;
        bool act = work && k + 1 < S && g < stop;
        if (act)
            rs.init(in_col, reinterpret_cast<const uint32_t *>(pay), pay_words, cbase >> 5,
                    (uint32_t)(cbase & 31) + g);
        uint32_t pos = g;
        while (__any_sync(0xffffffffu, act)) {
#pragma unroll
            for (int j = 0; j < kWindow; ++j) {
                if (act) {
                    if ((j & 1) == 0)
                        rs.refill();  // two table codes use at most 24 of > 32 bits
                    const uint32_t ent = lut[rs.peek12()];
                    uint32_t ns = ent >> 30, L = (ent >> 24) & 31u;
                    if (ns == 0) {  // longer than the table (rare)
                        rs.refill();
                        uint32_t sym;
                        if (!long_code(T, rs.buf64(), L, sym))
                            L = 1;
                        ns = 1;
                        rs.consume(L);
                        rs.refill();  // keep >= 12 bits for the next lookup
                    } else {
                        if (ns == 2) {
                            const uint32_t L0 = (ent >> 16) & 31u;
                            if (pos + L0 >= stop) {
                                ns = 1;
                                L = L0;
                            } else if (pos + L0 - g < 64) {
                                bmap |= 1ull << (pos + L0 - g);
                            }
                        }
                        rs.consume_small(L);
                    }
                    pos += L;
                    if (pos - g < 64)
                        bmap |= 1ull << (pos - g);
                    cnt1 += ns;
                    act = pos < stop;
                }
            }
            if (act)
                rs.top_up();
            cp_async_wait<2>();
        }
        cp_async_wait<0>();  // the ring is reused below
        e1 = pos;
    }
    uint32_t cnt = cnt1, e = e1;
    // 2. settle the entry points: all at once on the exits just counted,
    //    then again wherever an exit moved
    uint32_t entry = g;  // lane 0 already starts on the true path (g == 0)
    uint32_t used = g;
    bool first = true;
    for (;;) {
        const uint32_t pe = __shfl_up_sync(0xffffffffu, e, 1, S);
        const bool redo = work && k > 0 && (first || pe != used);
        if (!__any_sync(0xffffffffu, redo))
            break;
        if (redo) {
            used = pe;
            entry = pe;
            if (k + 1 < S)
                settle_segment(T, pay, pay_words, cbase, g, stop, entry, bmap, cnt1, e1, cnt,
                               e);
        }
        first = false;
    }
    // 3. output offsets: segmented exclusive scan of the counts
    const uint32_t own = (work && k + 1 < S) ? cnt : 0u;
    uint32_t x = own;
    for (uint32_t d = 1; d < S; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, d, S);
        if (k >= d)
            x += y;
    }
    const uint32_t O = x - own;
    uint32_t todo = 0;
    if (work && O < m)
        todo = (k + 1 == S) ? m - O : (own < m - O ? own : m - O);
    const bool final_seg = work && O < m && O + todo == m;

    // 4. decode on the true path and write the bytes
    {
        RingStream rs;
        bool act = todo > 0;
        uint8_t *const ob = si.out + c * cs;  // chunk output, 16-byte aligned
        const uint32_t qend = O + todo;
        uint32_t pos = entry, q = O, fl = O;  // q: next byte, fl: first unflushed byte
        if (act)
            rs.init(in_col, reinterpret_cast<const uint32_t *>(pay), pay_words, cbase >> 5,
                    (uint32_t)(cbase & 31) + entry);
        while (__any_sync(0xffffffffu, act)) {
            // a window far from the segment's end needs no per-code checks:
            // at most 16 symbols and 8 x 32 bits
            const bool easy = act && qend - q >= 2 * kWindow && lim - pos >= 32 * kWindow;
#pragma unroll
            for (int j = 0; j < kWindow; ++j) {
                if (act) {
                    if ((j & 1) == 0)
                        rs.refill();  // two table codes use at most 24 of > 32 bits
                    const uint32_t ent = lut[rs.peek12()];
                    uint32_t ns = ent >> 30, L = (ent >> 24) & 31u, sy = ent;
                    if (ns == 0) {  // longer than the table (rare)
                        rs.refill();
                        uint32_t sym = 0;
                        if (!long_code(T, rs.buf64(), L, sym)) {
                            bad = true;
                            L = 0;
                        }
                        ns = 1;
                        sy = sym;
                        if (!easy && pos + L > lim)
                            bad = true;
                        rs.consume(L);
                        rs.refill();  // keep >= 12 bits for the next lookup
                    } else {
                        if (!easy && ns == 2 && (qend - q < 2 || pos + L > lim)) {
                            ns = 1;
                            L = (ent >> 16) & 31u;
                        }
                        if (!easy && pos + L > lim)
                            bad = true;
                        rs.consume_small(L);
                    }
                    // both bytes always: an unused second byte is overwritten
                    // by the next symbol and never flushed
                    const uint32_t q1 = q + 1;
                    out_colb[((q & 31u) >> 2) * 128 + (q & 3u)] = (uint8_t)sy;
                    out_colb[((q1 & 31u) >> 2) * 128 + (q1 & 3u)] = (uint8_t)(sy >> 8);
                    q += ns;
                    pos += L;
                    if (!easy)
                        act = !bad && q < qend;
                }
            }
            if (easy)
                act = !bad && q < qend;
            if (act)
                rs.top_up();
            cp_async_wait<2>();
            // flush the half that holds `fl` once it is complete
            const uint32_t hs = fl & ~15u;
            if (!bad && q >= hs + 16) {
                if (fl == hs) {
                    const uint32_t *h = out_col + ((hs & 31u) >> 2) * 32;
                    *reinterpret_cast<uint4 *>(ob + hs) = make_uint4(h[0], h[32], h[64], h[96]);
                } else {
                    for (uint32_t b = fl; b < hs + 16; ++b)
                        ob[b] = out_colb[((b & 31u) >> 2) * 128 + (b & 3u)];
                }
                fl = hs + 16;
            }
        }
        cp_async_wait<0>();
        if (!bad) {
            for (uint32_t b = fl; b < q; ++b)
                ob[b] = out_colb[((b & 31u) >> 2) * 128 + (b & 3u)];
            if (todo && final_seg && c + 1 < chunks && pos != lim)
                bad = true;
        }
    }
    return __any_sync(0xffffffffu, bad);
}

}  // namespace dec
}  // namespace huff
