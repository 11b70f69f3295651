// Decoder device routines, shared by the single-stream kernel (decode.cu)
// and the batched kernel (batch.cu).  See decode.cu for the design.
#pragma once

#include "huff_internal.cuh"

namespace huff {
namespace dec {

constexpr int kLutBits = 12;
constexpr int kLutSize = 1 << kLutBits;
constexpr int kOutRing = 32;  // output ring: 128 bytes per lane (one 4 KiB-aligned block per warp)
// Input ring and window, by the ring's 16-byte cells per lane (C = 8: 4 KiB
// per warp, 32-lookup windows; C = 16: 8 KiB per warp, 64-lookup windows
// whose output is flushed after each 32 lookups)
template <int C> struct RingCfg {
    static constexpr int kInRing = 4 * C;   // words per lane
    static constexpr int kWindow = 4 * C;   // table lookups per unchecked window
    static constexpr int kInFlight = C / 2 - 1;  // groups left in flight at a window's end
};
constexpr int kCheckedWindow = 12;  // lookups per checked window
constexpr int kMaxPerLookup = 2;
constexpr uint32_t kFull = 0xffffffffu;

// Lookup table entry for a 12-bit window (first stream bit = MSB), 32 bits:
//   bits 24..31  s0, the byte of the first code in the window;
//   bits 16..23  s1, the byte of the second code when it also fits, else 0;
//   bits  8..15  8 * ns, ns = 1 or 2 codes;
//   bits  0..7   L, the total length of those codes (1..12);
// and 0 when the window starts with a code longer than 12 bits (or with no
// code at all).  The entry itself is the shift that drops the codes from
// the bit buffer (the wrap-mode funnel shifts read only its low five bits,
// and above bit 5 it is a multiple of 64), so the only work between two
// lookups of a lane is that shift, the next window's index and address.
// entry >> 8 is the output queue's operand: its low five bits are the shift
// 8 * ns and the entry's top 8 * ns bits are the symbols.  The length of
// the first code alone is in a second, byte-wide table.  The table is
// stored in C interleaved copies ([entry][copy]); lane l reads copy l mod C.
struct Tables {
    const uint32_t *lut;  // copy 0 of entry i at lut[i * copies]
    uint32_t copies;
    const uint8_t *len0;
    const uint32_t *count;
    const uint32_t *first;
    const uint32_t *start;
    const uint8_t *sorted;
    uint32_t max_len;
    __device__ __forceinline__ uint32_t entry(uint32_t idx) const { return lut[idx * copies]; }
};

// Shared-memory state of one stream's decode tables (C copies of the table).
template <int C>
struct DecodeShared {
    uint32_t lut[kLutSize * C];
    uint8_t len0[kLutSize];
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

// Shared-memory rings of one warp: input [word][lane] and output [row][lane]
// columns, the output block 4 KiB aligned (its wrap is one AND-OR).
struct WarpRings {
    uint32_t in_col;   // shared address of this lane's input column
    uint32_t out_col;  // shared address of this lane's output column
};

// Table entry of the 12-bit window at the top of bh, from this lane's copy
// (lut_l = copy base of this lane, stride = 4 * copies from the constant
// bank).  Volatile like the ring accesses, so that the order written below
// (each lookup's table load before the previous lookup's ring store) reaches
// the compiled code: a load cannot be moved above a shared store it might
// alias.
__device__ __forceinline__ uint32_t lut_ld(uint32_t lut_l, uint32_t stride, uint32_t bh)
{
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];"
                 : "=r"(v)
                 : "r"(imad(bh >> (32 - kLutBits), stride, lut_l)));
    return v;
}
// entry fields
__device__ __forceinline__ uint32_t ent_len(uint32_t e) { return e & 31u; }
__device__ __forceinline__ uint32_t ent_count(uint32_t e) { return (e >> 11) & 3u; }
__device__ __forceinline__ uint32_t len0_at(const uint8_t *len0, uint32_t bh)
{
    return len0[bh >> (32 - kLutBits)];
}

// Codes longer than the table: canonical search by length on a 32-bit window.
__device__ __forceinline__ bool long_code(const Tables &T, uint32_t v, uint32_t &L, uint32_t &sym)
{
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

// Bit reader over the payload's u32 words straight from global memory (used
// by the short settle walks).  Words come in blocks of four; the block after
// the current one is always in flight.  Words past the payload read as zero.
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

// 16-byte copy global -> shared, not kept in L1 (each lane streams its own
// chunk, so nothing is read twice through L1; measured on 1 GiB text the
// L1-allocating form took the decoder from 0.85 to 1.11 ms); bytes beyond
// `src_bytes` (0..16) are zero
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
                 "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Bit stream of one lane fed through its part of the warp's input ring.
// The ring holds, per lane, eight 16-byte cells of the payload as it lies in
// global memory (16-byte aligned groups of four words): cell c of lane l at
// byte c * 512 + l * 16 of the warp's 4 KiB-aligned block, so one 16-byte
// cp.async fills a cell and the 32 lanes' cells of a row are one 512-byte
// line of shared memory.  Words are numbered from w0, the payload word that
// holds the chunk's first bit; `ph` is the position of w0 in its group.
//
// The bit buffer bh:bl holds `have` valid bits, left-aligned.  `have` is
// kept in the low six bits of H (0 <= have <= 63); the bits above are junk:
// consume() subtracts a whole table word whose low five bits are the length,
// so the junk never reaches the low six bits, and the wrap-mode shifts read
// only the low five.
//
// Ring invariant (C cells of 4 words per lane): after every top-up more than
// 4C - 4 words are requested beyond the next one to read, in groups of 4,
// and the C/2 - 1 most recent groups may still be in flight; so the next
// 1 + 2C words have landed (C = 8: 17, C = 16: 33), and one window moves at
// most C + 7 + 1 words into the bit buffer (a checked window reads at most
// 12 codes of <= 32 bits, an unchecked one at most one such code and 4C of
// <= 12 bits plus one spare refill: 15 and 26 words; the buffer holds < 64
// bits).  Requests never reach the cell of a word that has not been read.
// Each top-up also asks L2 for the line 64 words past the requests.
template <int C>
struct BitsT {
    static constexpr int kInRing = 4 * C;
    uint32_t col;          // shared address of this lane's cell in row 0
    const uint4 *gp;       // the 16-byte group holding w0 (groups may start up to 3 words early)
    uint32_t g0lo;         // that group's index, low bits (its ring cell)
    uint32_t nfull;        // groups from gp that lie wholly inside the payload
    uint32_t tailb;        // payload bytes in group nfull (0..12)
    uint32_t ph;           // w0's position in its group
    uint32_t widx;    // next word to move into the bit buffer
    uint32_t fgr;     // next group to request, counted from g0
    uint32_t raddr;   // ring address of word widx
    uint32_t nxt;     // word widx, preloaded
    uint32_t bh, bl;  // bit buffer
    uint32_t H;       // have in the low six bits

    // ring address of word w (from w0)
    __device__ __forceinline__ uint32_t slot(uint32_t w) const
    {
        const uint32_t v = w + ph;
        return col + ((g0lo + (v >> 2)) & (C - 1u)) * 512 + (v & 3u) * 4;
    }
    // the address after ring address a: the next word of the cell, or the
    // first word of the next cell (a carry through the lane bits, set to all
    // ones, into the cell number), within the lane's C cells
    __device__ __forceinline__ uint32_t next_slot(uint32_t a, uint32_t k) const
    {
        return (imad(k, kc[kFour], a | 0x1f0u) & ((C - 1u) * 512u + 12u)) | col;
    }
    // request group fgr (four words), zero-filled past the payload
    __device__ __forceinline__ void fetch()
    {
        const uint32_t d = col + ((g0lo + fgr) & (C - 1u)) * 512;
        const uint32_t bytes = fgr < nfull ? 16u : (fgr == nfull ? tailb : 0u);
        cp_async16(d, bytes ? (const void *)(gp + fgr) : (const void *)gp, bytes);
        ++fgr;
        cp_async_commit();
    }
    __device__ __forceinline__ void top_up()
    {
        while (4 * fgr - (widx + ph) <= (uint32_t)kInRing - 4)
            fetch();
        if (fgr + 16 < nfull)  // ask L2 for the line 64 words past the requests
            asm volatile("prefetch.global.L2 [%0];" ::"l"(gp + fgr + 16));
    }
    // start at bit `pbit` counted from the first bit of payload word word0;
    // column: this lane's cell in row 0 of a (C * 512)-byte aligned block
    __device__ __forceinline__ void init(uint32_t column, const uint32_t *pay, uint64_t nw,
                                         uint64_t word0, uint32_t pbit)
    {
        col = column;
        const uint32_t lead = (uint32_t)(reinterpret_cast<uintptr_t>(pay) >> 2) & 3u;
        const uint4 *groups = reinterpret_cast<const uint4 *>(pay - lead);
        const uint64_t gend = nw + lead;  // virtual end: payload words + words before it in group 0
        const uint64_t v0 = word0 + lead;
        const uint64_t g0 = v0 >> 2;  // group holding w0
        gp = groups + g0;
        g0lo = (uint32_t)g0;
        const uint64_t full = gend >> 2;  // groups wholly inside the payload
        const uint64_t nf = full > g0 ? full - g0 : 0;
        nfull = nf < 0xffffffffull ? (uint32_t)nf : 0xffffffffu;
        tailb = 4 * (full >= g0 ? (uint32_t)(gend & 3) : 0u);  // the partial group full, if any
        ph = (uint32_t)(v0 & 3);
        widx = pbit >> 5;
        fgr = (widx + ph) >> 2;
#pragma unroll
        for (int r = 0; r < kInRing / 4; ++r)
            fetch();
        cp_async_wait<0>();
        const uint32_t sh = pbit & 31;
        raddr = slot(widx);
        bh = lds(raddr) << sh;
        bl = 0;
        H = 32 - sh;
        ++widx;
        raddr = next_slot(raddr, 1u);
        nxt = lds(raddr);
    }
    __device__ __forceinline__ uint32_t have() const { return H & 63u; }
    // stream bits consumed so far, counted from the first bit of word w0
    __device__ __forceinline__ uint32_t bitpos() const { return 32 * widx - have(); }
    // top the buffer up to at least 32 valid bits.  Straight-line code: k is
    // 1 when have < 32, else 0, every update is a multiply-add by k (the
    // buffer's free bits are zero, so adding is or-ing) and the next word is
    // loaded under a predicate.
    __device__ __forceinline__ void refill()
    {
        const uint32_t k = (~H >> 5) & 1u;
        bh = imad(k, __funnelshift_r(nxt, 0u, H), bh);  // nxt >> have
        bl = imad(k, __funnelshift_r(0u, nxt, H), bl);  // nxt << (32 - have), 0 at have = 0
        H = imad(k, kc[k32], H);
        widx = imad(k, kc[kOne], widx);
        raddr = next_slot(raddr, k);
        lds_if(k, raddr, nxt);
    }
    // drop the L = (t & 31) bits of t (a table entry: 1 <= L <= 12, 0 for a
    // long code); the rest of t is a multiple of 64 and never reaches have
    __device__ __forceinline__ void consume_t(uint32_t t)
    {
        bh = __funnelshift_l(bl, bh, t);
        bl = __funnelshift_l(0u, bl, t);
        H = imad(t, kc[kMinus1], H);
    }
    // drop L <= 32 bits
    __device__ __forceinline__ void consume(uint32_t L)
    {
        bh = __funnelshift_lc(bl, bh, L);
        bl = L >= 32 ? 0u : bl << L;
        H -= L;
    }
};

// Output bytes of one lane: a 64-bit queue in registers, oldest byte
// highest (big-endian), fed by the table entries' funnel shifts, and the
// lane's column of the warp's output ring (row r of lane l at byte
// r * 128 + 4 * l of the warp's 4 KiB-aligned block; kOutRing rows).  `P`
// counts the pending bits (a multiple of 8, < 64) in its low bits; adding a
// whole table entry adds 8 * ns there and junk only from bit 8 up.  `addr`
// is the ring slot of the word being filled.  store() writes that word every
// time it is called -- the four oldest pending bytes when P >= 32, else a
// partial word that a later store overwrites -- and moves to the next row
// when the word was complete, so it needs no predicate and no branch.
struct OutQ {
    uint32_t hi, lo;  // pending bytes in the low P bits of hi:lo
    uint32_t P;
    uint32_t addr;  // ring slot of the word being filled
    uint32_t base;  // 4 KiB-aligned base of the warp's output block
    uint32_t col;   // this lane's column (row 0)

    // the queue at output position q (the bytes of q's word before q are
    // placeholders, never flushed)
    __device__ __forceinline__ void start(uint32_t column, uint32_t q)
    {
        col = column;
        base = column & ~0xfffu;
        hi = lo = 0;
        P = (q & 3u) * 8;
        addr = column + ((q >> 2) & (kOutRing - 1)) * 128;
    }
    // append the top 8 * ns bits of table entry e (s = e >> 8: its low five
    // bits are 8 * ns, its higher ones land in P's junk)
    __device__ __forceinline__ void merge(uint32_t e)
    {
        const uint32_t sft = e >> 8;
        hi = __funnelshift_l(lo, hi, sft);
        lo = __funnelshift_l(e, lo, sft);
        P = imad(sft, kc[kOne], P);
    }
    __device__ __forceinline__ void store()
    {
        const uint32_t w = __funnelshift_r(lo, hi, P);  // bits [P - 32, P) when P >= 32
        sts(addr, __byte_perm(w, 0u, 0x0123));
        const uint32_t f = P & 32u;
        addr = ((imad(f, kc[kFour], addr)) & 0xfffu) | base;
        P = imad(f, kc[kMinus1], P);
    }
    // the pending bytes (< 4) as the word being filled, for the final flush
    __device__ __forceinline__ void store_partial()
    {
        const uint32_t p = P & 63u;
        sts(addr, __byte_perm(__funnelshift_lc(0u, lo, 32u - p), 0u, 0x0123));
    }
    // ring row of the word being filled (0..kOutRing-1) and pending bytes
    __device__ __forceinline__ uint32_t row() const { return ((addr - col) & 0xfffu) >> 7; }
    __device__ __forceinline__ uint32_t pending() const { return (P & 63u) >> 3; }
    __device__ __forceinline__ uint32_t byte_at(uint32_t b) const
    {
        return lds_u8(col + ((b >> 2) & (kOutRing - 1)) * 128 + (b & 3u));
    }
    __device__ __forceinline__ uint32_t word_row(uint32_t w) const
    {
        return lds(col + (w & (kOutRing - 1)) * 128);
    }
};

// Count codewords from bit `pos` (relative to the chunk's first bit `cbase`)
// until the first boundary at or past `stop`, from global memory.  Invalid
// bits (possible off the true path) count as 1-bit codewords.
__device__ __forceinline__ void count_codes(const Tables &T, const uint8_t *pay, uint64_t nw,
                                            uint64_t cbase, uint32_t pos, uint32_t stop,
                                            uint32_t &n, uint32_t &e)
{
    uint32_t cnt = 0;
    if (pos < stop) {
        Reader rd;
        rd.init(pay, nw, cbase + pos);
        while (pos < stop) {
            rd.refill();
            const uint32_t idx = (uint32_t)(rd.buf >> (64 - kLutBits));
            const uint32_t ent = T.entry(idx);
            uint32_t L = ent_len(ent), ns = ent_count(ent);
            if (ent == 0) {
                uint32_t sym;
                if (!long_code(T, (uint32_t)(rd.buf >> 32), L, sym))
                    L = 1;
                ns = 1;
            } else if (ns > 1 && pos + L >= stop) {  // later codes may start past stop
                L = T.len0[idx];
                ns = 1;
            }
            pos += L;
            cnt += ns;
            rd.consume(L);
        }
    }
    n = cnt;
    e = pos;
}

// Codeword boundaries seen in the first kSyncBits bits of a sub-segment's
// count (bit d set: a codeword starts d bits after the cut), kept in four
// named registers (the word is picked by selects, never by an array index,
// which would put the map in local memory).  256 bits: a Huffman decode
// started off the true path almost always rejoins it within that distance,
// so the settle walk below rarely has to recount a whole sub-segment.
constexpr uint32_t kSyncBits = 256;
struct SyncMap {
    uint64_t w0, w1, w2, w3;
    __device__ __forceinline__ void clear()
    {
        w0 = 1;  // the cut itself
        w1 = w2 = w3 = 0;
    }
    __device__ __forceinline__ void set(uint32_t d)
    {
        const uint64_t b = 1ull << (d & 63);
        const uint32_t j = d >> 6;
        w0 |= j == 0 ? b : 0;
        w1 |= j == 1 ? b : 0;
        w2 |= j == 2 ? b : 0;
        w3 |= j == 3 ? b : 0;
    }
    __device__ __forceinline__ uint64_t word(uint32_t j) const
    {
        return j == 0 ? w0 : j == 1 ? w1 : j == 2 ? w2 : w3;
    }
    __device__ __forceinline__ bool test(uint32_t d) const { return (word(d >> 6) >> (d & 63)) & 1; }
    // boundaries before d (d < kSyncBits)
    __device__ __forceinline__ uint32_t below(uint32_t d) const
    {
        const uint32_t j = d >> 6;
        return (j > 0 ? __popcll(w0) : 0) + (j > 1 ? __popcll(w1) : 0) + (j > 2 ? __popcll(w2) : 0) +
               __popcll(word(j) & ((1ull << (d & 63)) - 1));
    }
};

// Sub-segment [g, stop) was counted from g (cnt1 codewords, exit e1, early
// boundaries bmap).  Given its true entry point, walk the true path one
// codeword at a time until it lands on one of the recorded boundaries: from
// there both paths are the same codeword sequence, so only the codewords
// before the meeting point change.  If they do not meet within the recorded
// kSyncBits bits, recount from the entry point.
__device__ __forceinline__ void settle_segment(const Tables &T, const uint8_t *pay, uint64_t nw,
                                               uint64_t cbase, uint32_t g, uint32_t stop,
                                               uint32_t entry, const SyncMap &bmap, uint32_t cnt1,
                                               uint32_t e1, uint32_t &cnt, uint32_t &e)
{
    uint32_t pos = entry, steps = 0;
    Reader rd;
    bool started = false;
    for (;;) {
        const uint32_t d = pos - g;
        if (d < kSyncBits && bmap.test(d)) {  // met: same path from here on
            cnt = steps + cnt1 - bmap.below(d);
            e = e1;
            return;
        }
        if (pos >= stop) {  // left the sub-segment before meeting
            cnt = steps;
            e = pos;
            return;
        }
        if (d >= kSyncBits)
            break;
        if (!started) {
            rd.init(pay, nw, cbase + pos);
            started = true;
        }
        rd.refill();
        const uint32_t idx = (uint32_t)(rd.buf >> (64 - kLutBits));
        uint32_t L = T.len0[idx];  // first code only: every boundary matters
        if (T.entry(idx) == 0) {
            uint32_t sym;
            if (!long_code(T, (uint32_t)(rd.buf >> 32), L, sym))
                L = 1;
        }
        pos += L;
        ++steps;
        rd.consume(L);
    }
    count_codes(T, pay, nw, cbase, entry, stop, cnt, e);
}

// Validate the stream header and build the decode tables of one stream in
// shared memory (all NT threads of the CTA take part; `reporter` writes *d_n
// and the header errors).  `scratch` is shared memory for kLutSize u16 that
// is free while the tables are built.  Returns true when there are chunks to
// decode.
// The CTA barrier, as the barrier of prepare's thread group.
struct CtaSync {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

// Validate a stream's header and build its tables, by a group of NT threads
// (tid = 0..NT-1) whose barrier is sync().
template <int NT, int C, class Sync>
__device__ __forceinline__ bool prepare(const uint8_t *stream_in, uint64_t bytes, uint8_t *out,
                                        uint64_t cap, unsigned long long *d_n, int32_t *status,
                                        bool reporter, DecodeShared<C> &sh, uint16_t *scratch,
                                        StreamInfo &si, int tid, Sync sync)
{
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
    sync();
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
    sync();
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
    sync();
    for (int b = tid; b < 256; b += NT) {
        const uint32_t L = sh.len_s[b];
        if (L) {
            uint32_t r = 0;
            for (int j = 0; j < b; ++j)
                r += sh.len_s[j] == L;
            sh.sorted[sh.start[L] + r] = (uint8_t)b;
        }
    }
    sync();
    // pass 1: the first code of every 12-bit window, sym | L << 8 (0: none)
    const uint32_t lut_len = max_len < (uint32_t)kLutBits ? max_len : (uint32_t)kLutBits;
    for (int v = tid; v < kLutSize; v += NT) {
        uint32_t ent = 0;
        for (uint32_t L = 1; L <= lut_len; ++L) {
            const uint32_t c = (uint32_t)v >> (kLutBits - L);
            if (sh.count[L] && c - sh.first[L] < sh.count[L]) {
                ent = sh.sorted[sh.start[L] + c - sh.first[L]] | (L << 8);
                break;
            }
        }
        scratch[v] = (uint16_t)ent;
    }
    sync();
    // pass 2: append the second code when it also fits in the window
    for (int v = tid; v < kLutSize; v += NT) {
        const uint32_t e0 = scratch[v];
        uint32_t ent = 0, first_len = 0;
        if (e0) {
            const uint32_t L0 = e0 >> 8;
            ent = ((e0 & 0xffu) << 24) | (8u << 8) | L0;
            if (L0 < (uint32_t)kLutBits) {
                const uint32_t e1 = scratch[((uint32_t)v << L0) & (kLutSize - 1)];
                const uint32_t L1 = e1 >> 8;
                if (e1 && L0 + L1 <= (uint32_t)kLutBits)
                    ent = ((e0 & 0xffu) << 24) | ((e1 & 0xffu) << 16) | (16u << 8) | (L0 + L1);
            }
            first_len = L0;
        }
#pragma unroll
        for (int c = 0; c < C; ++c)
            sh.lut[v * C + c] = ent;
        sh.len0[v] = (uint8_t)first_len;
    }
    sync();

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
    si.T.copies = C;
    si.T.len0 = sh.len0;
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

// Store the complete 16-byte groups of [fl, q) from the output ring.
__device__ __forceinline__ void flush_groups(uint8_t *ob, const OutQ &ow, uint32_t &fl, uint32_t q)
{
    uint32_t hs = fl & ~15u;
    while (q >= hs + 16) {
        if (fl == hs) {
            const uint32_t w = hs >> 2;
            *reinterpret_cast<uint4 *>(ob + hs) =
                make_uint4(ow.word_row(w), ow.word_row(w + 1), ow.word_row(w + 2), ow.word_row(w + 3));
        } else {
            for (uint32_t b = fl; b < hs + 16; ++b)
                ob[b] = (uint8_t)ow.byte_at(b);
        }
        hs += 16;
        fl = hs;
    }
}

// Store the complete 32-byte groups of [fl, q) from the output ring, for an
// output ob that is 32-byte aligned: one 256-bit store per group, so each
// lane's write is a whole sector (measured on 1 GiB text: 0.87 -> 0.80 ms
// against 16-byte groups).
__device__ __forceinline__ void flush_groups32(uint8_t *ob, const OutQ &ow, uint32_t &fl, uint32_t q)
{
    uint32_t hs = fl & ~31u;
    while (q >= hs + 32) {
        if (fl == hs) {
            const uint32_t w = hs >> 2;
            asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(ob + hs),
                         "r"(ow.word_row(w)), "r"(ow.word_row(w + 1)), "r"(ow.word_row(w + 2)),
                         "r"(ow.word_row(w + 3)), "r"(ow.word_row(w + 4)), "r"(ow.word_row(w + 5)),
                         "r"(ow.word_row(w + 6)), "r"(ow.word_row(w + 7))
                         : "memory");
        } else {
            for (uint32_t b = fl; b < hs + 32; ++b)
                ob[b] = (uint8_t)ow.byte_at(b);
        }
        hs += 32;
        fl = hs;
    }
}

// Decode warp task `task` of stream si with S lanes per chunk (32/S chunks
// per warp).  in_col / out_col: shared addresses of this lane's columns of
// the warp's rings (the output block 4 KiB aligned).  Returns true
// (warp-uniform) if the stream is corrupt.  kWhole: S == 1, one lane per
// chunk, compiled without the count / settle / scan phases.
template <bool kWhole, int C>
__device__ __forceinline__ bool decode_task_s(const StreamInfo &si, uint32_t S_arg, uint64_t task,
                                              uint32_t in_s, uint32_t out_s)
{
    constexpr int kWindow = RingCfg<C>::kWindow;
    constexpr int kInFlight = RingCfg<C>::kInFlight;
    const uint32_t S = kWhole ? 1u : S_arg;
    const Tables &T = si.T;
    const int lane = threadIdx.x & 31;
    const uint32_t lut_l = smem_u32(T.lut) + ((uint32_t)lane & (T.copies - 1)) * 4;
    const uint32_t stride = T.copies == 1 ? kc[kFour] : T.copies == 2 ? kc[kEight] : kc[k16];
    const uint8_t *len0 = T.len0;
    const uint64_t n = si.n, chunks = si.chunks, pbits = si.pbits, pay_words = si.pay_words;
    const uint32_t cs = si.cs;
    const uint64_t *offs = si.offs;
    const uint8_t *pay = si.pay;
    const uint32_t G = 32 / S;
    const uint32_t k = (uint32_t)lane & (S - 1);
    const uint32_t grp = (uint32_t)lane / S;
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
    const uint32_t *pw = reinterpret_cast<const uint32_t *>(pay);
    const uint32_t b0 = (uint32_t)(cbase & 31);  // chunk bit 0 within word w0

    // 1. count each sub-segment but the last from its cut point
    uint32_t cnt1 = 0, e1 = g;
    SyncMap bmap;
    bmap.clear();
    if (S > 1) {  // uniform: every lane of the warp takes this branch
        BitsT<C> rs = {};
        bool act = work && k + 1 < S && g < stop;
        if (act)
            rs.init(in_s, pw, pay_words, cbase >> 5, b0 + g);
        uint32_t pos = g;
        // 1a. code by code through the first kSyncBits bits, recording the
        //     boundaries
        bool head = act;
        while (__any_sync(kFull, head)) {
            if (head) {
                rs.refill();
                uint32_t L = len0_at(len0, rs.bh);
                if (L == 0) {
                    uint32_t sym;
                    if (!long_code(T, rs.bh, L, sym))
                        L = 1;
                }
                rs.consume(L);
                rs.refill();
                pos += L;
                ++cnt1;
                if (pos - g < kSyncBits)
                    bmap.set(pos - g);
                head = pos - g < kSyncBits && pos < stop;
                act = pos < stop;
            }
        }
        // 1b. windows of table lookups, several codes per lookup
        uint32_t cnt8 = 0;  // 8 x codes
        while (__any_sync(kFull, act)) {
            // an unchecked window reads at most one long code plus kWindow
            // table lookups of <= 12 bits
            const bool easy = stop - pos >= 32 + kLutBits * kWindow;
            if (__all_sync(kFull, easy || !act)) {
                if (act) {
                    rs.refill();
                    if (lut_ld(lut_l, stride, rs.bh) == 0) {  // a long code (rare)
                        uint32_t L, sym;
                        if (!long_code(T, rs.bh, L, sym))
                            L = 1;
                        rs.consume(L);
                        rs.refill();
                        cnt8 += 8;
                    }
                }
#pragma unroll
                for (int j = 0; j < kWindow; ++j) {
                    if (act) {
                        if ((j & 1) == 0 && j > 0)
                            rs.refill();  // two lookups use at most 24 of >= 32 bits
                        // a long code's entry is all zero: the lane stays on
                        // it for the rest of the window
                        const uint32_t ent = lut_ld(lut_l, stride, rs.bh);
                        rs.consume_t(ent);
                        cnt8 += (ent >> 8) & 24u;
                    }
                }
            } else {
#pragma unroll 1
                for (int j = 0; j < kCheckedWindow; ++j) {
                    if (act) {
                        rs.refill();
                        uint32_t L = len0_at(len0, rs.bh);  // one code at a time
                        if (L == 0) {
                            uint32_t sym;
                            if (!long_code(T, rs.bh, L, sym))
                                L = 1;
                        }
                        rs.consume(L);
                        cnt8 += 8;
                        act = rs.bitpos() - b0 < stop;
                    }
                }
            }
            if (act) {
                pos = rs.bitpos() - b0;
                act = pos < stop;
            }
            if (act)
                rs.top_up();
            cp_async_wait<kInFlight>();
        }
        cp_async_wait<0>();  // the ring is reused below
        if (work && k + 1 < S && g < stop) {
            cnt1 += cnt8 >> 3;
            e1 = rs.bitpos() - b0;
        }
    }
    uint32_t cnt = cnt1, e = e1;
    // 2. settle the entry points: all at once on the exits just counted,
    //    then again wherever an exit moved
    uint32_t entry = g;  // lane 0 already starts on the true path (g == 0)
    uint32_t used = g;
    bool first = true;
    for (;;) {
        const uint32_t pe = __shfl_up_sync(kFull, e, 1, S);
        const bool redo = work && k > 0 && (first || pe != used);
        if (!__any_sync(kFull, redo))
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
        const uint32_t y = __shfl_up_sync(kFull, x, d, S);
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
        BitsT<C> rs = {};
        OutQ ow;
        bool act = todo > 0;
        uint8_t *const ob = si.out + c * cs;  // chunk output, 16-byte aligned
        const bool wide = (reinterpret_cast<uintptr_t>(ob) & 31u) == 0;
        const uint32_t qend = O + todo;
        uint32_t pos = entry, q = O, fl = O;  // q: next byte, fl: first unflushed byte
        ow.start(out_s, O);
        if (act)
            rs.init(in_s, pw, pay_words, cbase >> 5, b0 + entry);
        while (__any_sync(kFull, act)) {
            // far from the segment's end a window needs no per-code checks:
            // at most 2 * kWindow symbols and kWindow x 12 bits, plus one
            // long code.  The unchecked window runs only when every lane of
            // the warp is in that state, so it needs no per-lane predicate
            // either.
            const bool easy = act && qend - q >= 1 + kMaxPerLookup * kWindow &&
                              lim - pos >= 32 + kLutBits * kWindow;
            uint32_t q0 = q, row0 = ow.row(), p0 = ow.pending();
            if (__all_sync(kFull, easy)) {
                rs.refill();
                if (lut_ld(lut_l, stride, rs.bh) == 0) {  // a long code (rare)
                    uint32_t L = 0, sym = 0;
                    if (!long_code(T, rs.bh, L, sym)) {
                        bad = true;  // nothing more is flushed
                        act = false;
                    }
                    rs.consume(L);
                    rs.refill();
                    ow.merge((sym << 24) | (8u << 8));
                    ow.store();
                }
                // A long code's entry is all zero, so it consumes and emits
                // nothing: the lane stays on it for the rest of the window
                // and resolves it at the start of the next.  Pairs of
                // lookups: a refill (>= 32 bits) serves both, as two lookups
                // use at most 24 bits, and one store serves both, as the
                // queue then holds at most 3 + 2 * 2 bytes.  Software
                // pipelined: lookup j+1's table load is issued before lookup
                // j's bytes are queued.  The last pair's refill and table
                // load for a lookup beyond the window are harmless (one more
                // word at most, within the ring bound).
                uint32_t ent = lut_ld(lut_l, stride, rs.bh);
#pragma unroll 1
                for (int half = 0; half < kWindow / 32; ++half) {
#pragma unroll 4
                    for (int p = 0; p < 16; ++p) {
                        rs.consume_t(ent);
                        const uint32_t ent1 = lut_ld(lut_l, stride, rs.bh);
                        ow.merge(ent);
                        rs.consume_t(ent1);
                        rs.refill();
                        ent = lut_ld(lut_l, stride, rs.bh);
                        ow.merge(ent1);
                        ow.store();
                    }
                    if (half + 1 < kWindow / 32) {
                        // a 64-lookup window flushes after its first 32 lookups
                        // (at most 65 bytes and 17 rows so far), so the output
                        // ring never holds more than one half's bytes
                        const uint32_t qm = q0 + 4 * ((ow.row() - row0) & (kOutRing - 1)) +
                                            ow.pending() - p0;
                        if (!bad) {
                            if (wide)
                                flush_groups32(ob, ow, fl, qm);
                            else
                                flush_groups(ob, ow, fl, qm);
                        }
                        q0 = qm;
                        row0 = ow.row();
                        p0 = ow.pending();
                    }
                }
            } else {
#pragma unroll 1
                for (int j = 0; j < kCheckedWindow; ++j) {
                    if (act) {
                        rs.refill();
                        const uint32_t ent = lut_ld(lut_l, stride, rs.bh);
                        uint32_t L, ns, y;
                        if (ent == 0) {
                            uint32_t sym = 0;
                            L = 0;
                            if (!long_code(T, rs.bh, L, sym))
                                bad = true;
                            ns = 1;
                            y = (sym << 24) | (8u << 8);
                        } else {
                            L = ent_len(ent);
                            ns = ent_count(ent);
                            y = ent;
                            if (q + ns > qend || pos + L > lim) {  // first code only
                                L = len0_at(len0, rs.bh);
                                ns = 1;
                                y = (ent & 0xff000000u) | (8u << 8);
                            }
                        }
                        if (pos + L > lim)
                            bad = true;
                        if (!bad) {
                            rs.consume(L);
                            ow.merge(y);
                            ow.store();
                            q += ns;
                            pos += L;
                        }
                        act = !bad && q < qend;
                    }
                }
            }
            // bytes queued in this window: whole rows stored plus the change
            // in pending bytes (a window moves fewer than kOutRing rows)
            q = q0 + 4 * ((ow.row() - row0) & (kOutRing - 1)) + ow.pending() - p0;
            pos = rs.bitpos() - b0;
            if (act) {
                act = q < qend;
                if (act)
                    rs.top_up();
            }
            cp_async_wait<kInFlight>();
            if (!bad) {
                if (wide)
                    flush_groups32(ob, ow, fl, q);
                else
                    flush_groups(ob, ow, fl, q);
            }
        }
        cp_async_wait<0>();
        if (!bad) {
            if (todo)
                ow.store_partial();  // the bytes of the word being filled
            if (wide)
                flush_groups32(ob, ow, fl, q);
            for (uint32_t b = fl; b < q; ++b)
                ob[b] = (uint8_t)ow.byte_at(b);
            if (todo && final_seg && c + 1 < chunks && pos != lim)
                bad = true;
        }
    }
    return __any_sync(kFull, bad);
}

// C: input ring cells per lane (8: 32-lookup windows; 16: 64-lookup windows
// and twice the input ring)
template <int C = 8>
__device__ __forceinline__ bool decode_task(const StreamInfo &si, uint32_t S, uint64_t task,
                                            uint32_t in_s, uint32_t out_s)
{
    return S == 1 ? decode_task_s<true, C>(si, 1, task, in_s, out_s)
                  : decode_task_s<false, C>(si, S, task, in_s, out_s);
}

}  // namespace dec
}  // namespace huff
