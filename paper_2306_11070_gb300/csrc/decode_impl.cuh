// Decoder device routines, shared by the single-stream kernel (decode.cu)
// and the batched kernel (batch.cu).  See decode.cu for the design.
#pragma once

#include "huff_internal.cuh"

namespace huff {
namespace dec {

constexpr int kLutBits = 12;
constexpr int kLutSize = 1 << kLutBits;
constexpr int kInRing = 32;   // input ring: words per lane
constexpr int kOutRing = 32;  // output ring: 128 bytes per lane
constexpr int kWindow = 32;   // table lookups per unchecked window
constexpr int kCheckedWindow = 12;  // lookups per checked window
constexpr int kMaxPerLookup = 3;
constexpr uint32_t kFull = 0xffffffffu;

// Lookup table entry for a 12-bit window (first stream bit = MSB), 32 bits:
//   bits  0..23  the bytes of up to three whole codes in the window, first
//                code in the low byte, zero above the last one;
//   bits 24..29  L, the total length of those codes (1..12);
//   bits 30..31  ns, their number (1..3);
// and 0 when the window starts with a code longer than 12 bits (or with no
// code at all).  So entry >> 24 = L + 64 * ns: its low five bits are L, as a
// wrap-mode funnel shift wants them, and the rest is a multiple of 64.  The
// length of the first code alone is in a second, byte-wide table.
struct Tables {
    const uint32_t *lut;
    const uint8_t *len0;
    const uint32_t *count;
    const uint32_t *first;
    const uint32_t *start;
    const uint8_t *sorted;
    uint32_t max_len;
};

// Shared-memory state of one stream's decode tables.
struct DecodeShared {
    uint32_t lut[kLutSize];
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

// table entry of the 12-bit window at the top of bh.  Volatile like the ring
// accesses, so that the order written below (each lookup's table load
// before the previous lookup's ring store) reaches the compiled code:
// a load cannot be moved above a shared store it might alias.
__device__ __forceinline__ uint32_t lut_ld(uint32_t lut_s, uint32_t bh)
{
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(imad(bh >> (32 - kLutBits), kc[kFour], lut_s)));
    return v;
}
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

__device__ __forceinline__ void cp_async4(uint32_t dst, const uint32_t *src, bool valid)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src),
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
// w0, the payload word that holds the chunk's first bit.
//
// The bit buffer bh:bl holds `have` valid bits, left-aligned.  `have` is
// kept in the low six bits of H (0 <= have <= 63); the bits above are junk:
// consume() subtracts a whole table word whose low five bits are the length,
// so the junk never reaches the low six bits, and the wrap-mode shifts read
// only the low five.
//
// Ring invariant: after every top-up more than kInRing - 4 words are
// requested beyond the next one to read, in groups of 4, and the three most
// recent groups may still be in flight; so the next 1 + 16 words have
// landed, and one window moves at most 15 words into the bit buffer (a
// checked window reads at most 12 codes of <= 32 bits, an unchecked one at
// most one such code and 32 of <= 12 bits plus one spare refill, and the
// buffer holds < 64 bits).
// Requests never reach the slot of a word that has not been read.  Each
// top-up also asks L2 for the line 64 words past the requests.
struct Bits {
    uint32_t col;           // shared address of this lane's column
    const uint32_t *words;  // payload
    uint64_t nwords;
    uint64_t w0;
    uint32_t widx;    // next word to move into the bit buffer
    uint32_t fidx;    // next word to request
    uint32_t nxt;     // word widx, preloaded
    uint32_t bh, bl;  // bit buffer
    uint32_t H;       // have in the low six bits

    __device__ __forceinline__ uint32_t slot(uint32_t w) const { return col + (w & (kInRing - 1)) * 128; }
    // request words fidx .. fidx+3 (fidx is a multiple of 4, so they fill
    // ring rows (fidx & 31) .. +3 without wrapping)
    __device__ __forceinline__ void fetch4()
    {
        const uint32_t d = slot(fidx);
        const uint64_t aw = w0 + fidx;
        if (aw + 4 <= nwords) {
            const uint32_t *src = words + aw;
            cp_async4(d, src, true);
            cp_async4(d + 128, src + 1, true);
            cp_async4(d + 256, src + 2, true);
            cp_async4(d + 384, src + 3, true);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const bool ok = aw + j < nwords;
                cp_async4(d + 128 * j, words + (ok ? aw + j : 0), ok);
            }
        }
        fidx += 4;
        cp_async_commit();
    }
    __device__ __forceinline__ void top_up()
    {
        while (fidx - widx <= (uint32_t)kInRing - 4)
            fetch4();
        const uint64_t pf = w0 + fidx + 64;
        if (pf < nwords)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(words + pf));
    }
    // start at bit `pbit` counted from the first bit of word w0
    __device__ __forceinline__ void init(uint32_t column, const uint32_t *pay, uint64_t nw,
                                         uint64_t word0, uint32_t pbit)
    {
        col = column;
        words = pay;
        nwords = nw;
        w0 = word0;
        widx = pbit >> 5;
        fidx = widx & ~3u;
#pragma unroll
        for (int r = 0; r < kInRing / 4; ++r)
            fetch4();
        cp_async_wait<0>();
        const uint32_t sh = pbit & 31;
        bh = lds(slot(widx)) << sh;
        bl = 0;
        H = 32 - sh;
        ++widx;
        nxt = lds(slot(widx));
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
        lds_if(k, imad(widx & (kInRing - 1), kc[k128], col), nxt);
    }
    // drop the L = (t & 31) bits of t = entry >> 24 (1 <= L <= 31); the rest
    // of t is a multiple of 64 and never reaches have
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

// Output bytes of one lane assembled in a register and stored to its column
// of the warp's output ring one completed word at a time (row r of lane l at byte
// r * 128 + 4 * l of the warp's ring; the ring holds kOutRing words).
// `lo` holds the bytes of the word being filled at its low end, `sh` = 8 *
// (bytes in lo) and R = 128 * (number of the word being filled), of which
// the row is R mod (128 * kOutRing).  Bytes above the filled ones are zero,
// so appending is adding.
struct OutWord {
    uint32_t col;  // shared address of this lane's column
    uint32_t lo, sh, R;

    __device__ __forceinline__ void start(uint32_t column, uint32_t q)
    {
        col = column;
        lo = 0;
        sh = (q & 3u) * 8;
        R = (q >> 2) * 128;
    }
    __device__ __forceinline__ uint32_t addr() const
    {
        return imad(R & ((kOutRing - 1) * 128), kc[kOne], col);
    }
    // append the ns bytes of y (zero above them); a completed word is stored
    __device__ __forceinline__ void emit(uint32_t y, uint32_t ns)
    {
        const uint32_t hi = __funnelshift_l(y, 0u, sh);  // y >> (32 - sh), 0 at sh = 0
        lo = imad(y, 1u << sh, lo);                      // lo | y << sh
        sh = imad(ns, kc[kEight], sh);
        const uint32_t full = sh >> 5;                   // the word is complete
        sts_if(full, addr(), lo);
        lo = imad(full, imad(lo, kc[kMinus1], hi), lo);  // full ? hi : lo
        R = imad(full, kc[k128], R);
        sh = imad(full, kc[kMinus32], sh);
    }
    // output position, given the position q0 and value R0 of R at some
    // earlier point
    __device__ __forceinline__ uint32_t pos_from(uint32_t q0, uint32_t R0) const
    {
        return ((q0 >> 2) + ((R - R0) >> 7)) * 4 + (sh >> 3);
    }
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
            const uint32_t ent = T.lut[idx];
            uint32_t L = (ent >> 24) & 31u, ns = ent >> 30;
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
        if (T.lut[idx] == 0) {
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
template <int NT>
__device__ __forceinline__ bool prepare(const uint8_t *stream_in, uint64_t bytes, uint8_t *out,
                                        uint64_t cap, unsigned long long *d_n, int32_t *status,
                                        bool reporter, DecodeShared &sh, uint16_t *scratch,
                                        StreamInfo &si)
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
    __syncthreads();
    // pass 2: append the following codes while they fit in the window
    for (int v = tid; v < kLutSize; v += NT) {
        const uint32_t e0 = scratch[v];
        uint32_t ent = 0, first_len = 0;
        if (e0) {
            const uint32_t L0 = e0 >> 8;
            uint32_t syms = e0 & 0xffu, tot = L0, ns = 1;
#pragma unroll
            for (int k = 1; k < kMaxPerLookup; ++k) {
                if (ns == (uint32_t)k && tot < (uint32_t)kLutBits) {
                    const uint32_t e1 = scratch[((uint32_t)v << tot) & (kLutSize - 1)];
                    const uint32_t L1 = e1 >> 8;
                    if (e1 && tot + L1 <= (uint32_t)kLutBits) {
                        syms |= (e1 & 0xffu) << (8 * k);
                        tot += L1;
                        ++ns;
                    }
                }
            }
            ent = syms | (tot << 24) | (ns << 30);
            first_len = L0;
        }
        sh.lut[v] = ent;
        sh.len0[v] = (uint8_t)first_len;
    }
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
__device__ __forceinline__ void flush_groups(uint8_t *ob, const OutWord &ow, uint32_t &fl,
                                             uint32_t q)
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

// Decode warp task `task` of stream si with S lanes per chunk (32/S chunks
// per warp).  in_col / out_col: this lane's column of the warp's rings.
// Returns true (warp-uniform) if the stream is corrupt.  kWhole: S == 1, one
// lane per chunk, compiled without the count / settle / scan phases.
template <bool kWhole>
__device__ __forceinline__ bool decode_task_s(const StreamInfo &si, uint32_t S_arg, uint64_t task,
                                              uint32_t *in_col, uint32_t *out_col)
{
    const uint32_t S = kWhole ? 1u : S_arg;
    const Tables &T = si.T;
    const uint32_t lut_s = smem_u32(T.lut);
    const uint8_t *len0 = T.len0;
    const uint32_t in_s = smem_u32(in_col), out_s = smem_u32(out_col);
    const uint64_t n = si.n, chunks = si.chunks, pbits = si.pbits, pay_words = si.pay_words;
    const uint32_t cs = si.cs;
    const uint64_t *offs = si.offs;
    const uint8_t *pay = si.pay;
    const int lane = threadIdx.x & 31;
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
        Bits rs = {};
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
        uint32_t cnt = 0;
        while (__any_sync(kFull, act)) {
            // an unchecked window reads at most one long code plus 16 table
            // lookups of <= 12 bits
            const bool easy = stop - pos >= 32 + kLutBits * kWindow;
            if (__all_sync(kFull, easy || !act)) {
                if (act) {
                    rs.refill();
                    if (lut_ld(lut_s, rs.bh) == 0) {  // a long code (rare)
                        uint32_t L, sym;
                        if (!long_code(T, rs.bh, L, sym))
                            L = 1;
                        rs.consume(L);
                        rs.refill();
                        ++cnt;
                    }
                }
#pragma unroll
                for (int j = 0; j < kWindow; ++j) {
                    if (act) {
                        if ((j & 1) == 0 && j > 0)
                            rs.refill();  // two lookups use at most 24 of >= 32 bits
                        // a long code's entry is all zero: the lane stays on
                        // it for the rest of the window
                        const uint32_t ent = lut_ld(lut_s, rs.bh);
                        rs.consume_t(ent >> 24);
                        cnt += ent >> 30;
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
                        ++cnt;
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
            cp_async_wait<3>();
        }
        cp_async_wait<0>();  // the ring is reused below
        if (work && k + 1 < S && g < stop) {
            cnt1 += cnt;
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
        Bits rs = {};
        OutWord ow = {};
        bool act = todo > 0;
        uint8_t *const ob = si.out + c * cs;  // chunk output, 16-byte aligned
        const uint32_t qend = O + todo;
        uint32_t pos = entry, q = O, fl = O;  // q: next byte, fl: first unflushed byte
        ow.start(out_s, O);
        if (act)
            rs.init(in_s, pw, pay_words, cbase >> 5, b0 + entry);
        while (__any_sync(kFull, act)) {
            // far from the segment's end a window needs no per-code checks:
            // at most 3 * 16 symbols and 16 x 32 bits.  The unchecked window
            // runs only when every lane of the warp is in that state, so it
            // needs no per-lane predicate either.
            // A window reads at most one long code (resolved first) plus 16
            // table lookups of <= 12 bits and 3 symbols each.
            const bool easy = act && qend - q >= 1 + kMaxPerLookup * kWindow &&
                              lim - pos >= 32 + kLutBits * kWindow;
            const uint32_t q0 = q, R0 = ow.R;
            if (__all_sync(kFull, easy)) {
                rs.refill();
                if (lut_ld(lut_s, rs.bh) == 0) {  // a long code (rare)
                    uint32_t L = 0, sym = 0;
                    if (!long_code(T, rs.bh, L, sym)) {
                        bad = true;  // nothing more is flushed
                        act = false;
                    }
                    rs.consume(L);
                    rs.refill();
                    ow.emit(sym, 1);
                }
                // A long code's entry is all zero, so it consumes and emits
                // nothing: the lane stays on it for the rest of the window
                // and resolves it at the start of the next.  Software
                // pipelined: lookup j+1's table load is issued before lookup
                // j's output is appended.
                // Pairs of lookups: a refill (>= 32 bits) serves both, as
                // two lookups use at most 24 bits.  The last pair's refill
                // and table load for a lookup beyond the window are
                // harmless (one more word at most, within the ring bound).
                uint32_t ent = lut_ld(lut_s, rs.bh);
#pragma unroll 4
                for (int p = 0; p < kWindow / 2; ++p) {
                    const uint32_t t0 = ent >> 24;
                    rs.consume_t(t0);
                    const uint32_t ent1 = lut_ld(lut_s, rs.bh);
                    ow.emit(imad(t0, kc[kMinusTop8], ent), t0 >> 6);  // the symbol bytes
                    const uint32_t t1 = ent1 >> 24;
                    rs.consume_t(t1);
                    rs.refill();
                    ent = lut_ld(lut_s, rs.bh);
                    ow.emit(imad(t1, kc[kMinusTop8], ent1), t1 >> 6);
                }
            } else {
#pragma unroll 1
                for (int j = 0; j < kCheckedWindow; ++j) {
                    if (act) {
                        rs.refill();
                        const uint32_t ent = lut_ld(lut_s, rs.bh);
                        uint32_t L, ns8, y;
                        if (ent == 0) {
                            rs.refill();
                            uint32_t sym = 0;
                            L = 0;
                            if (!long_code(T, rs.bh, L, sym))
                                bad = true;
                            ns8 = 8;
                            y = sym;
                        } else {
                            L = (ent >> 24) & 31u;
                            ns8 = (ent >> 30) << 3;
                            y = ent & 0xffffffu;
                            if (q + (ns8 >> 3) > qend || pos + L > lim) {  // first code only
                                L = len0_at(len0, rs.bh);
                                ns8 = 8;
                                y &= 0xffu;
                            }
                        }
                        if (pos + L > lim)
                            bad = true;
                        if (!bad) {
                            rs.consume(L);
                            ow.emit(y, ns8 >> 3);
                            q += ns8 >> 3;
                            pos += L;
                        }
                        act = !bad && q < qend;
                    }
                }
            }
            q = ow.pos_from(q0, R0);
            pos = rs.bitpos() - b0;
            if (act) {
                act = q < qend;
                if (act)
                    rs.top_up();
            }
            cp_async_wait<3>();
            if (!bad)
                flush_groups(ob, ow, fl, q);
        }
        cp_async_wait<0>();
        if (!bad) {
            if (todo)
                sts(ow.addr(), ow.lo);  // bytes carried over by the last emit
            for (uint32_t b = fl; b < q; ++b)
                ob[b] = (uint8_t)ow.byte_at(b);
            if (todo && final_seg && c + 1 < chunks && pos != lim)
                bad = true;
        }
    }
    return __any_sync(kFull, bad);
}

__device__ __forceinline__ bool decode_task(const StreamInfo &si, uint32_t S, uint64_t task,
                                            uint32_t *in_col, uint32_t *out_col)
{
    return S == 1 ? decode_task_s<true>(si, 1, task, in_col, out_col)
                  : decode_task_s<false>(si, S, task, in_col, out_col);
}

}  // namespace dec
}  // namespace huff
