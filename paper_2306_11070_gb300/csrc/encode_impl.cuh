// Encoder device routines, shared by the single-stream kernel (encode.cu)
// and the fused batched kernel (batch.cu).  See encode.cu for the design.
#pragma once

#include "huff_internal.cuh"

namespace huff {
namespace enc {

constexpr int kTblWords = 256 * 32;  // [byte][lane] table, 32 KiB
// fast path (codes of at most kFastMaxLen bits): 32 symbols per lane and
// step, 1024 per warp step, 16 steps per unit
constexpr int kFastSyms = 32;
constexpr int kFastStep = 32 * kFastSyms;
constexpr int kFastSteps = kUnitSymbols / kFastStep;
// the low 10 bits of a sum of 32 entries are the sum of their lengths while
// every length is at most 22 (the code sits above bit 9 of its entry)
constexpr uint32_t kFastMaxLen = 22;
constexpr uint32_t kSumMask = 1023;
// long codes (23..32 bits): 16 symbols per lane and step
constexpr int kLongSyms = 16;
constexpr int kLongStep = 32 * kLongSyms;
constexpr int kLongSteps = kUnitSymbols / kLongStep;
// warp buffer: a guard word, then the words of one step (a fast step writes
// at most 1024 x 22 / 32 = 704 words after the < 32 carried bits, a long one
// 512 x 32 / 32 = 512), rounded up
constexpr int kWarpObuf = 1 + kFastStep * (int)kFastMaxLen / 32 + 15;  // 720 words

// One stream being written: input, unit offsets, output layout.
struct Job {
    const uint8_t *in;
    uint64_t n;
    uint32_t cs;
    const unsigned long long *unit_off;  // exclusive bit prefix per unit, total at [units]
    uint64_t units;
    uint8_t *out;
    uint64_t out_cap;
    uint64_t pay0;  // payload byte offset
    uint64_t cap_words;
    bool table_fits;
};

__device__ __forceinline__ Job make_job(const uint8_t *in, uint64_t n, uint32_t cs,
                                        const unsigned long long *unit_off, uint8_t *out,
                                        uint64_t out_cap)
{
    Job j;
    j.in = in;
    j.n = n;
    j.cs = cs;
    j.unit_off = unit_off;
    j.units = (n + kUnitSymbols - 1) / kUnitSymbols;
    j.out = out;
    j.out_cap = out_cap;
    const uint64_t chunks = n ? ceil_div_u64(n, cs) : 0;
    j.pay0 = kHeaderBytes + 8 * chunks;
    j.table_fits = j.pay0 <= out_cap;
    j.cap_words = j.table_fits ? (out_cap - j.pay0) / 4 : 0;
    return j;
}

// Codes per emit check in the fast path: floor(32 / longest), as a template.
__device__ __forceinline__ int emit_group(uint32_t max_len)
{
    const uint32_t gq = max_len ? 32u / max_len : 16u;
    return gq >= 16 ? 16 : gq >= 8 ? 8 : gq >= 4 ? 4 : gq >= 3 ? 3 : gq >= 2 ? 2 : 1;
}

// Header (threads 0..255 of the calling CTA) and the stream size.
__device__ __forceinline__ void write_header(const Job &J, const huff_codebook_t *cb,
                                             unsigned long long *out_bytes, int32_t *status)
{
    const int tid = threadIdx.x;
    if (J.out_cap >= kHeaderBytes) {
        if (tid < 256)
            J.out[tid] = cb->len[tid];
        if (tid == 0) {
            *reinterpret_cast<uint64_t *>(J.out + 256) = J.n;
            *reinterpret_cast<uint32_t *>(J.out + 264) = J.cs;
            *reinterpret_cast<uint32_t *>(J.out + 268) = cb->max_len;
        }
    }
    if (tid == 0) {
        const uint64_t total = J.units ? J.unit_off[J.units] : 0;
        *out_bytes = J.pay0 + 4 * ((total + 31) >> 5);
        if (!J.table_fits)
            set_status(status, HUFF_ERR_CAPACITY);
    }
}

// Entry of the fast table at shared address a (the table is read-only
// while units are encoded).
__device__ __forceinline__ uint32_t tbl_at(uint32_t a)
{
    uint32_t v;
    asm("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}

// Per-lane replicated code table (16-byte aligned), built by threads tid =
// 0..nt-1 (by default all threads of the CTA).  Fast entry = (code << (32 -
// len)) | len: the code left-aligned, its length in the low bits, zeros
// between them (len <= 22 leaves bits 5..9 clear).  A thread per byte reads
// its length and code once and fills the byte's 32 lane copies with eight
// 16-byte stores, rotated by the byte so that the stores of a warp spread
// over all eight 16-byte bank groups.
__device__ __forceinline__ void build_table(const huff_codebook_t *cb, uint32_t *tbl, bool fast,
                                            int tid = threadIdx.x, int nt = blockDim.x)
{
    if (fast) {
        for (int b = tid; b < 256; b += nt) {
            const uint32_t L = cb->len[b];
            const uint32_t e = L ? (cb->code[b] << (32 - L)) | L : 0u;
            const uint4 v = make_uint4(e, e, e, e);
            uint4 *row = reinterpret_cast<uint4 *>(tbl + b * 32);
#pragma unroll
            for (int j = 0; j < 8; ++j)
                row[(j + b) & 7] = v;
        }
    } else {
        for (int i = tid; i < 256 * 16; i += nt) {
            const int b = i >> 4;
            tbl[i] = cb->code[b];
            tbl[256 * 16 + i] = cb->len[b];
        }
    }
}

// Zero this warp's buffer (kWarpObuf words at wob); every step leaves the
// words it used zero again, so this runs once per unit.
__device__ __forceinline__ void clear_buffer(uint32_t *wob, int lane)
{
    for (int j = lane; j < kWarpObuf; j += 32)
        wob[j] = 0u;
    __syncwarp();
}

template <int N>
__device__ __forceinline__ uint32_t byte_of(const uint32_t (&w)[N], int k)
{
    return __byte_perm(w[k >> 2], 0u, 0x4440u | (uint32_t)(k & 3));
}

__device__ __forceinline__ void red_or(uint32_t a, uint32_t v)
{
    asm volatile("red.shared.or.b32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

// Pack the 32 codes of one lane (fast entries e, sums sc at every emit
// check) into the warp's word buffer, the lane's bits starting at bit p0.
// hi:lo holds the lane's last 64 bits.  With G = floor(32 / longest) codes
// between checks, at most one word boundary is crossed per check; each check
// writes the last completed word (its bits of this lane: bits of this lane
// that were not yet shifted in are zero), so a word is written once or, with
// the same bits, again.  A check before the lane's first word is complete
// writes zeros to the word before it (the guard word for lane 0).
//  - kSts (a full step: every lane has 32 codes, so at least 32 bits):
//    plain stores.  Such a zero word can only land on the previous lane's
//    last complete word, and only at a check before the last one, while
//    that lane writes the word again at its last check; so every complete
//    word ends with its owner's value, with no atomics and no clearing.
//  - otherwise a lane may have no bits at all: OR into a zeroed buffer.
// Returns the end of the lane's bits and its last partial word (zero bits
// when there is none), high-aligned.
template <int G, bool kSts>
__device__ __forceinline__ uint32_t pack32(const uint32_t (&e)[kFastSyms],
                                           const uint32_t (&sc)[(kFastSyms + G - 1) / G], uint32_t p0,
                                           uint32_t wob_s, uint32_t &part)
{
    uint32_t hi = 0u, lo = 0u, E = p0;
#pragma unroll
    for (int k = 0; k < kFastSyms; ++k) {
        const uint32_t x = e[k];
        hi = __funnelshift_l(lo, hi, x);  // (hi:lo) <<= len
        lo = __funnelshift_l(x, lo, x);   //   ... | code
        if ((k + 1) % G == 0 || k == kFastSyms - 1) {
            E = p0 + (sc[k / G] & kSumMask);  // end of the lane's bits so far
            const uint32_t a = imad(E >> 5, kc[kFour], wob_s - 4), v = __funnelshift_r(lo, hi, E);
            if (kSts)
                sts(a, v);
            else
                red_or(a, v);
        }
    }
    part = __funnelshift_lc(0u, lo, 32u - (E & 31u));
    return E;
}

// The last r (< 32) bits of the code stream before symbol `base` (> 0), as the
// high bits of a word: lane l re-codes byte base-1-l.  Warp-uniform result.
__device__ __forceinline__ uint32_t seam_word(const uint8_t *in, uint64_t base, uint32_t r,
                                              const uint32_t *tbl, bool fast, int lane)
{
    const uint32_t b = in[base - 1 - lane];
    uint32_t L, code;
    if (fast) {
        const uint32_t x = tbl[(b << 5) | lane];
        L = x & 31u;
        code = L ? x >> (32 - L) : 0u;
    } else {
        code = tbl[(b << 4) | (lane & 15)];
        L = tbl[256 * 16 + ((b << 4) | (lane & 15))];
    }
    uint32_t sfx = L;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, sfx, d);
        if (lane >= d)
            sfx += v;
    }
    const uint32_t before = sfx - L;  // bits between this code's end and base
    const uint32_t part = (L && before < r) ? code << (32 - r + before) : 0u;
    return __reduce_or_sync(0xffffffffu, part);
}

// Shared per-unit state of the encoders below.
struct UnitState {
    uint64_t base;   // first symbol of the unit
    uint64_t gbit;   // stream bit of the next step's first symbol
    uint32_t carry;  // bits of the partial word before the step, high-aligned
    uint32_t lead;   // distance from the step start to the next chunk start
    uint64_t next_chunk;  // index of that chunk
};

__device__ __forceinline__ UnitState unit_start(const Job &J, uint64_t u, const uint32_t *tbl,
                                                bool fast, int lane)
{
    UnitState st;
    st.base = u * kUnitSymbols;
    st.gbit = J.unit_off[u];
    st.carry = (st.base > 0 && (st.gbit & 31))
                   ? seam_word(J.in, st.base, (uint32_t)(st.gbit & 31), tbl, fast, lane)
                   : 0u;
    const uint32_t umod = (uint32_t)(st.base % J.cs);
    st.lead = umod ? J.cs - umod : 0u;
    st.next_chunk = (st.base + st.lead) / J.cs;
    return st;
}

// This lane's SPT input bytes of the step starting at symbol sb (m of them
// real, the rest zero), read straight from the input (partial steps only).
template <int SPT>
__device__ __forceinline__ int step_input_tail(const Job &J, uint64_t sb, int lane,
                                               uint32_t (&w)[SPT / 4])
{
    const uint64_t i0 = sb + (uint64_t)lane * SPT;
    const int m = i0 >= J.n ? 0 : (J.n - i0 >= (uint64_t)SPT ? SPT : (int)(J.n - i0));
#pragma unroll
    for (int j = 0; j < SPT / 4; ++j)
        w[j] = 0u;
#pragma unroll
    for (int k = 0; k < SPT; ++k)
        if (k < m)
            w[k >> 2] |= (uint32_t)J.in[i0 + k] << (8 * (k & 3));
    return m;
}

// Inclusive warp scan of the lanes' bit counts: (exclusive position, total).
__device__ __forceinline__ void scan_bits(uint32_t bits, int lane, uint32_t &pos, uint32_t &total)
{
    uint32_t incl = bits;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d)
            incl += v;
    }
    pos = incl - bits;
    total = __shfl_sync(0xffffffffu, incl, 31);
}

// Chunk offsets: the stream bit of every chunk that starts at one of this
// lane's symbols.  A chunk starts at a multiple of cs, itself a multiple of
// 16, so only at lane offset 0 or 16 (mid16: the bits of the lane's first 16
// symbols; only used when SPT = 32).
template <int SPT, int STEP>
__device__ __forceinline__ void step_chunks(const Job &J, const UnitState &st, uint64_t sb, int lane,
                                            uint32_t pos, uint32_t mid16)
{
    if (!J.table_fits)
        return;
    uint64_t *offs = reinterpret_cast<uint64_t *>(J.out + kHeaderBytes);
#pragma unroll
    for (int off = 0; off < SPT; off += 16) {
        const uint32_t d = (uint32_t)lane * SPT + off;
        const uint64_t bit = st.gbit + pos + (off ? mid16 : 0u);
        if (J.cs >= (uint32_t)STEP) {  // at most one start per step
            stg64_if(d == st.lead && sb + d < J.n, offs + st.next_chunk, bit);
        } else if (d >= st.lead && (d - st.lead) % J.cs == 0 && sb + d < J.n) {
            offs[(sb + d) / J.cs] = bit;
        }
    }
}

template <int STEP>
__device__ __forceinline__ void step_advance(const Job &J, UnitState &st, uint32_t step_bits)
{
    st.gbit += step_bits;
    if (st.lead >= (uint32_t)STEP) {
        st.lead -= STEP;
    } else if (J.cs >= (uint32_t)STEP) {
        st.lead = J.cs - (STEP - st.lead);
        ++st.next_chunk;
    } else {
        st.lead = (J.cs - (STEP - st.lead) % J.cs) % J.cs;
    }
}

// Whole words of the step out (coalesced); the partial last word is carried
// into the next step, or left to the next unit's seam at the unit end.
// kChecked: bound checks against the output capacity (else the words surely
// fit) and every word read cleared again for the next step's OR-ing.
// Returns true on overflow.
template <bool kChecked>
__device__ __forceinline__ bool step_output(const Job &J, UnitState &st, bool last, uint32_t step_bits,
                                            uint32_t *wob, int lane)
{
    uint32_t *pay = reinterpret_cast<uint32_t *>(J.out + J.pay0);
    const uint32_t r = (uint32_t)(st.gbit & 31);
    const uint32_t nw = (r + step_bits + 31) >> 5;
    const uint32_t tail = (r + step_bits) & 31u;
    const uint32_t nwrite = (last || tail == 0) ? nw : nw - 1;
    const uint64_t wbase = st.gbit >> 5;
    bool overflow = false;
    const uint32_t carry = tail ? wob[nw - 1] : 0u;
    if (!kChecked || wbase + nwrite <= J.cap_words) {
        for (uint32_t j0 = 0; j0 < nw; j0 += 32) {
            const uint32_t j = j0 + lane;
            const uint32_t v = j < nw ? wob[j] : 0u;
            stg_if(j < nwrite, pay + wbase + j, v);
            if (kChecked && j < nw)
                wob[j] = 0u;
        }
    } else {
        for (uint32_t j = lane; j < nw; j += 32) {
            if (j < nwrite) {
                if (wbase + j < J.cap_words)
                    pay[wbase + j] = wob[j];
                else
                    overflow = true;
            }
            wob[j] = 0u;
        }
    }
    st.carry = carry;
    return overflow;
}

// One 1024-symbol step of the fast encoder (codes of at most 22 bits, G =
// floor(32 / longest)).  kInner: the step lies inside the input, the unit
// is not the last one and its words fit the output, so the step needs none
// of the bound checks; its 32 input bytes per lane (w) were loaded ahead.
template <int G, bool kInner>
__device__ __forceinline__ bool fast_step(const Job &J, UnitState &st, int step, int lane,
                                          uint32_t tcol_s, uint32_t wob_s, uint32_t *wob,
                                          const uint32_t (&w)[8])
{
    constexpr int NC = (kFastSyms + G - 1) / G;
    const uint64_t sb = st.base + (uint64_t)step * kFastStep;
    int m = kFastSyms;
    uint32_t tw[8];
    if (kInner) {
#pragma unroll
        for (int j = 0; j < 8; ++j)
            tw[j] = w[j];
    } else {
        m = step_input_tail<kFastSyms>(J, sb, lane, tw);
    }

    // table entries of this lane's symbols; s accumulates whole entries,
    // whose low 10 bits sum the lengths
    uint32_t e[kFastSyms], sc[NC];
    uint32_t s = 0, mid16 = 0;
#pragma unroll
    for (int k = 0; k < kFastSyms; ++k) {
        e[k] = tbl_at(imad(byte_of(tw, k), kc[k128], tcol_s));
        if (!kInner && k >= m)
            e[k] = 0u;
        s = imad(e[k], kc[kOne], s);
        if ((k + 1) % G == 0 || k == kFastSyms - 1)
            sc[k / G] = s;
        if (k == 15)
            mid16 = s & kSumMask;
    }
    const uint32_t bits = s & kSumMask;
    uint32_t pos, step_bits;
    scan_bits(bits, lane, pos, step_bits);
    const uint32_t p0 = (uint32_t)(st.gbit & 31) + pos;

    step_chunks<kFastSyms, kFastStep>(J, st, sb, lane, pos, mid16);
    uint32_t part;
    if (kInner) {
        // complete words by plain stores, then each lane ORs its last partial
        // word into the next lane's first word (the last lane stores it: no
        // lane writes that word), and lane 0 ORs the carried bits into word 0
        const uint32_t E = pack32<G, true>(e, sc, p0, wob_s, part);
        __syncwarp();
        const uint32_t pa = imad(E >> 5, kc[kFour], wob_s);
        if (lane == 31)
            sts(pa, part);
        else
            red_or(pa, part);
        if (lane == 0)
            red_or(wob_s, st.carry);
    } else {
        // word 0 starts with the carried bits; every other word is zero
        sts_if(lane == 0, wob_s, st.carry);
        __syncwarp();
        const uint32_t E = pack32<G, false>(e, sc, p0, wob_s, part);
        red_or(imad(E >> 5, kc[kFour], wob_s), part);
    }
    __syncwarp();
    const bool last = sb + kFastStep >= J.n;
    const bool overflow = step_output<!kInner>(J, st, last, step_bits, wob, lane);
    __syncwarp();
    step_advance<kFastStep>(J, st, step_bits);
    return overflow;
}

__device__ __forceinline__ void load32(const uint8_t *p, uint32_t (&w)[8])
{
    const uint4 a = ld_stream16(p), b = ld_stream16(p + 16);
    w[0] = a.x;
    w[1] = a.y;
    w[2] = a.z;
    w[3] = a.w;
    w[4] = b.x;
    w[5] = b.y;
    w[6] = b.z;
    w[7] = b.w;
}

// Encode unit u of job J with the calling warp, codes of at most 22 bits.
// wob is the warp's buffer of kWarpObuf words (word 0 is the guard), tbl the
// CTA's table.  Returns true if a payload word fell outside the output
// capacity.
template <int G>
__device__ __forceinline__ bool encode_unit_fast(const Job &J, uint64_t u, const uint32_t *tbl,
                                                 uint32_t *wob)
{
    const int lane = threadIdx.x & 31;
    const uint32_t tcol_s = smem_u32(tbl + lane), wob_s = smem_u32(wob + 1);
    UnitState st = unit_start(J, u, tbl, true, lane);
    const bool inner = st.base + kUnitSymbols < J.n && (J.unit_off[u + 1] >> 5) < J.cap_words;
    if (!inner)
        clear_buffer(wob, lane);
    bool overflow = false;
    if (inner) {  // warp-uniform
        const uint8_t *p = J.in + st.base + lane * kFastSyms;
        uint32_t w[8];
        load32(p, w);
        for (int step = 0; step < kFastSteps; ++step) {
            uint32_t nx[8];
            if (step + 1 < kFastSteps)
                load32(p + (step + 1) * kFastStep, nx);  // one step ahead
            fast_step<G, true>(J, st, step, lane, tcol_s, wob_s, wob + 1, w);
#pragma unroll
            for (int j = 0; j < 8; ++j)
                w[j] = nx[j];
        }
    } else {
        const uint32_t none[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int step = 0; step < kFastSteps; ++step) {
            if (st.base + (uint64_t)step * kFastStep >= J.n)
                break;  // warp-uniform
            overflow |= fast_step<G, false>(J, st, step, lane, tcol_s, wob_s, wob + 1, none);
        }
    }
    return overflow;
}

// ---- codes gathered by multiply-add (single-stream encoder) ----------------
// The fast path above spends two funnel shifts per code on the ALU pipe,
// which bounds it.  Here a group of codes is gathered on the FMA pipe: the
// table holds (code, 2^len) per byte and lane, and a = a * 2^len + code
// appends a code to the group's bits; a starts at 1, so its leading one
// marks the group's length (a group has at most 31 bits).  Only the group
// then pays the funnel shifts into the 64-bit window and the emit check:
// per code one byte extract, one table load (8 bytes) and one IMAD, per
// group a leading-one search and three funnel shifts.  The groups of a lane
// are cut at its 16th symbol too, where a chunk may start.  Same stream,
// bit for bit.
constexpr int kTbl2Words = 256 * 32 * 2;  // [byte][lane] (code, 2^len), 64 KiB

__device__ __forceinline__ void build_table2(const huff_codebook_t *cb, uint32_t *tbl2)
{
    for (int i = threadIdx.x; i < 256 * 32; i += blockDim.x) {
        const int b = i >> 5;
        const uint32_t L = cb->len[b];
        tbl2[2 * i] = L ? cb->code[b] : 0u;
        tbl2[2 * i + 1] = 1u << L;  // 2^0 = 1 for a byte without a code: no bits
    }
}

// Codes per group: floor(31 / longest), as a template (31: the marker bit).
__device__ __forceinline__ int mad_group(uint32_t max_len)
{
    const uint32_t gq = max_len ? 31u / max_len : 16u;
    return gq >= 16 ? 16 : gq >= 8 ? 8 : gq >= 4 ? 4 : gq >= 3 ? 3 : gq >= 2 ? 2 : 1;
}

// As seam_word, from the (code, 2^len) table.
__device__ __forceinline__ uint32_t seam_word2(const uint8_t *in, uint64_t base, uint32_t r,
                                               const uint32_t *tbl2, int lane)
{
    const uint32_t b = in[base - 1 - lane];
    const uint2 x = reinterpret_cast<const uint2 *>(tbl2)[(b << 5) | lane];
    const uint32_t L = 31u - __clz(x.y), code = x.x;
    uint32_t sfx = L;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, sfx, d);
        if (lane >= d)
            sfx += v;
    }
    const uint32_t before = sfx - L;
    const uint32_t part = (L && before < r) ? code << (32 - r + before) : 0u;
    return __reduce_or_sync(0xffffffffu, part);
}

__device__ __forceinline__ UnitState unit_start2(const Job &J, uint64_t u, const uint32_t *tbl2,
                                                 int lane)
{
    UnitState st;
    st.base = u * kUnitSymbols;
    st.gbit = J.unit_off[u];
    st.carry = (st.base > 0 && (st.gbit & 31)) ? seam_word2(J.in, st.base, (uint32_t)(st.gbit & 31), tbl2, lane)
                                               : 0u;
    const uint32_t umod = (uint32_t)(st.base % J.cs);
    st.lead = umod ? J.cs - umod : 0u;
    st.next_chunk = (st.base + st.lead) / J.cs;
    return st;
}

// One 1024-symbol step (codes of at most 22 bits; G codes per group).
template <int G, bool kInner>
__device__ __forceinline__ bool mad_step(const Job &J, UnitState &st, int step, int lane,
                                         uint32_t tcol_s, uint32_t wob_s, uint32_t *wob,
                                         const uint32_t (&w)[8])
{
    constexpr int NH = (16 + G - 1) / G;  // groups per 16 symbols
    constexpr int NG = 2 * NH;
    const uint64_t sb = st.base + (uint64_t)step * kFastStep;
    int m = kFastSyms;
    uint32_t tw[8];
    if (kInner) {
#pragma unroll
        for (int j = 0; j < 8; ++j)
            tw[j] = w[j];
    } else {
        m = step_input_tail<kFastSyms>(J, sb, lane, tw);
    }
    uint32_t acc[NG], lg[NG];
    uint32_t bits = 0, mid16 = 0;
#pragma unroll
    for (int g = 0; g < NG; ++g) {
        const int k0 = (g / NH) * 16 + (g % NH) * G;
        uint32_t a = 1u;
#pragma unroll
        for (int j = 0; j < G; ++j) {
            const int k = k0 + j;
            if ((g % NH) * G + j < 16 && (kInner || k < m)) {
                uint2 x;
                asm("ld.shared.v2.u32 {%0, %1}, [%2];"
                    : "=r"(x.x), "=r"(x.y)
                    : "r"(imad(byte_of(tw, k), kc[k128] * 2u, tcol_s)));
                a = a * x.y + x.x;
            }
        }
        acc[g] = a;
        lg[g] = 31u - __clz(a);
        bits += lg[g];
        if (g == NH - 1)
            mid16 = bits;
    }
    uint32_t pos, step_bits;
    scan_bits(bits, lane, pos, step_bits);
    const uint32_t p0 = (uint32_t)(st.gbit & 31) + pos;
    step_chunks<kFastSyms, kFastStep>(J, st, sb, lane, pos, mid16);
    if (!kInner) {
        sts_if(lane == 0, wob_s, st.carry);  // word 0 starts with the carried bits
        __syncwarp();
    }
    // groups into the 64-bit window hi:lo, the last completed word out after
    // each group (see pack32 for why plain stores are enough when every
    // lane has 32 codes)
    // A group that crosses no word boundary would store the same word again:
    // only groups that cross one store (about one group in 2.4 on text),
    // which keeps the warp-buffer stores off the L1 data pipe.
    uint32_t hi = 0u, lo = 0u, E = p0;
#pragma unroll
    for (int g = 0; g < NG; ++g) {
        const uint32_t L = lg[g];
        const uint32_t top = __funnelshift_lc(0u, acc[g], 32u - L);  // the group's bits, high-aligned
        hi = __funnelshift_l(lo, hi, L);
        lo = __funnelshift_l(top, lo, L);
        const uint32_t E0 = E;
        E = imad(L, kc[kOne], E);
        if ((E ^ E0) >> 5) {  // a word was completed
            const uint32_t ad = imad(E >> 5, kc[kFour], wob_s - 4), v = __funnelshift_r(lo, hi, E);
            if (kInner)
                sts(ad, v);
            else
                red_or(ad, v);
        }
    }
    const uint32_t part = __funnelshift_lc(0u, lo, 32u - (E & 31u));
    if (kInner) {
        __syncwarp();
        const uint32_t pa = imad(E >> 5, kc[kFour], wob_s);
        if (lane == 31)
            sts(pa, part);
        else
            red_or(pa, part);
        if (lane == 0)
            red_or(wob_s, st.carry);
    } else {
        red_or(imad(E >> 5, kc[kFour], wob_s), part);
    }
    __syncwarp();
    const bool last = sb + kFastStep >= J.n;
    const bool overflow = step_output<!kInner>(J, st, last, step_bits, wob, lane);
    __syncwarp();
    step_advance<kFastStep>(J, st, step_bits);
    return overflow;
}

template <int G>
__device__ __forceinline__ bool encode_unit_mad(const Job &J, uint64_t u, const uint32_t *tbl2,
                                                uint32_t *wob)
{
    const int lane = threadIdx.x & 31;
    const uint32_t tcol_s = smem_u32(tbl2 + 2 * lane), wob_s = smem_u32(wob + 1);
    UnitState st = unit_start2(J, u, tbl2, lane);
    const bool inner = st.base + kUnitSymbols < J.n && (J.unit_off[u + 1] >> 5) < J.cap_words;
    if (!inner)
        clear_buffer(wob, lane);
    bool overflow = false;
    if (inner) {  // warp-uniform
        const uint8_t *p = J.in + st.base + lane * kFastSyms;
        uint32_t w[8];
        load32(p, w);
        for (int step = 0; step < kFastSteps; ++step) {
            uint32_t nx[8];
            if (step + 1 < kFastSteps)
                load32(p + (step + 1) * kFastStep, nx);  // one step ahead
            mad_step<G, true>(J, st, step, lane, tcol_s, wob_s, wob + 1, w);
#pragma unroll
            for (int j = 0; j < 8; ++j)
                w[j] = nx[j];
        }
    } else {
        const uint32_t none[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int step = 0; step < kFastSteps; ++step) {
            if (st.base + (uint64_t)step * kFastStep >= J.n)
                break;  // warp-uniform
            overflow |= mad_step<G, false>(J, st, step, lane, tcol_s, wob_s, wob + 1, none);
        }
    }
    return overflow;
}

// group: mad_group of the longest code, at least 3 (longer codes keep the
// funnel-shift path, where a group of one or two codes saves nothing)
__device__ __forceinline__ bool encode_unit_mad_g(const Job &J, uint64_t u, const uint32_t *tbl2,
                                                  int group, uint32_t *wob)
{
    switch (group) {
    case 16: return encode_unit_mad<16>(J, u, tbl2, wob);
    case 8: return encode_unit_mad<8>(J, u, tbl2, wob);
    case 4: return encode_unit_mad<4>(J, u, tbl2, wob);
    default: return encode_unit_mad<3>(J, u, tbl2, wob);
    }
}

// The same for codes of up to 32 bits: split code / length tables, 16
// symbols per lane and a 64-bit accumulator (rare: only very skewed inputs
// have codes this long).
__device__ __forceinline__ bool encode_unit_long(const Job &J, uint64_t u, const uint32_t *tbl,
                                                 uint32_t *wob_all)
{
    const int lane = threadIdx.x & 31;
    clear_buffer(wob_all, lane);
    uint32_t *wob = wob_all + 1;
    bool overflow = false;
    UnitState st = unit_start(J, u, tbl, false, lane);
    for (int step = 0; step < kLongSteps; ++step) {
        const uint64_t sb = st.base + (uint64_t)step * kLongStep;
        if (sb >= J.n)
            break;  // warp-uniform
        uint32_t w[4];
        const int m = step_input_tail<kLongSyms>(J, sb, lane, w);
        uint32_t e[kLongSyms], l2[kLongSyms];
        uint32_t bits = 0;
        const int col = lane & 15;
#pragma unroll
        for (int k = 0; k < kLongSyms; ++k) {
            const uint32_t b = byte_of(w, k);
            e[k] = k < m ? tbl[(b << 4) | col] : 0u;
            l2[k] = k < m ? tbl[256 * 16 + ((b << 4) | col)] : 0u;
            bits += l2[k];
        }
        uint32_t pos, step_bits;
        scan_bits(bits, lane, pos, step_bits);
        const uint32_t r = (uint32_t)(st.gbit & 31);
        if (lane == 0)
            wob[0] = st.carry;  // word 0 starts with the carried bits
        __syncwarp();
        step_chunks<kLongSyms, kLongStep>(J, st, sb, lane, pos, 0u);
        if (m > 0) {
            uint32_t wi = (r + pos) >> 5, nb = (r + pos) & 31u;
            uint64_t acc = 0;
#pragma unroll
            for (int k = 0; k < kLongSyms; ++k) {
                const uint32_t L = l2[k];
                acc = L ? ((acc << L) | e[k]) : acc;
                nb += L;
                if (nb >= 32) {
                    nb -= 32;
                    atomicOr(wob + wi, (uint32_t)(acc >> nb));
                    ++wi;
                }
            }
            if (nb)
                atomicOr(wob + wi, (uint32_t)acc << (32 - nb));
        }
        __syncwarp();
        overflow |= step_output<true>(J, st, sb + kLongStep >= J.n, step_bits, wob, lane);
        __syncwarp();
        step_advance<kLongStep>(J, st, step_bits);
    }
    return overflow;
}

__device__ __forceinline__ bool encode_unit(const Job &J, uint64_t u, const uint32_t *tbl, bool fast,
                                           int group, uint32_t *wob)
{
    if (!fast)
        return encode_unit_long(J, u, tbl, wob);
    switch (group) {
    case 16: return encode_unit_fast<16>(J, u, tbl, wob);
    case 8: return encode_unit_fast<8>(J, u, tbl, wob);
    case 4: return encode_unit_fast<4>(J, u, tbl, wob);
    case 3: return encode_unit_fast<3>(J, u, tbl, wob);
    case 2: return encode_unit_fast<2>(J, u, tbl, wob);
    default: return encode_unit_fast<1>(J, u, tbl, wob);
    }
}

}  // namespace enc
}  // namespace huff
