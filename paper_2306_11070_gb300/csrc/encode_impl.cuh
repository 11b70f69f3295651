// Encoder device routines, shared by the single-stream kernel (encode.cu)
// and the fused batched kernel (batch.cu).  See encode.cu for the design.
#pragma once

#include "huff_internal.cuh"

namespace huff {
namespace enc {

constexpr int kSymsPerThread = 16;
constexpr int kStepSyms = 32 * kSymsPerThread;          // 512 per warp step
constexpr int kStepsPerUnit = kUnitSymbols / kStepSyms;  // 32
constexpr int kTblWords = 256 * 32;                      // 32 KiB
constexpr int kWarpObuf = kStepSyms + 8;                 // 32-bit codes + alignment
constexpr int kFastMaxLen = 24;

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

// Per-lane replicated code table (all threads of the CTA take part).
__device__ __forceinline__ void build_table(const huff_codebook_t *cb, uint32_t *tbl, bool fast)
{
    if (fast) {
        for (int i = threadIdx.x; i < kTblWords; i += blockDim.x) {
            const int b = i >> 5;
            const uint32_t L = cb->len[b];
            tbl[i] = L ? (cb->code[b] << (32 - L)) | L : 0u;
        }
    } else {
        for (int i = threadIdx.x; i < 256 * 16; i += blockDim.x) {
            const int b = i >> 4;
            tbl[i] = cb->code[b];
            tbl[256 * 16 + i] = cb->len[b];
        }
    }
}

__device__ __forceinline__ uint32_t byte_of(const uint32_t (&w)[4], int k)
{
    return __byte_perm(w[k >> 2], 0u, 0x4440u | (uint32_t)(k & 3));
}

// A word of the warp buffer, written under a predicate without a branch:
// OR-ed when `shared` (the word also holds another lane's bits), else stored.
__device__ __forceinline__ void put_word(uint32_t f, uint32_t shared, uint32_t a, uint32_t v)
{
    asm volatile("{\n\t.reg .pred p, q, ps, pn;\n\t"
                 "setp.ne.u32 p, %2, 0;\n\t"
                 "setp.ne.u32 q, %3, 0;\n\t"
                 "and.pred ps, p, q;\n\t"
                 "and.pred pn, p, !q;\n\t"
                 "@pn st.shared.u32 [%0], %1;\n\t"
                 "@ps red.shared.or.b32 [%0], %1;\n\t}"
                 ::"r"(a), "r"(v), "r"(f), "r"(shared)
                 : "memory");
}

// Append the 16 codes of one lane (fast table entries, len <= 24) at bit p0
// of the warp's word-aligned buffer (shared address wob).  s[k] is the
// total length of codes 0..k.  With G = floor(32 / longest code), G codes
// always fit beside fewer than 32 pending bits in the 64-bit accumulator,
// so a word can complete only at every G-th code; the check there is
// straight-line code.  Words are whole and owned by this lane except the
// first one when p0 is not word aligned (it holds the end of the previous
// lane's bits) and the final partial one: those two are OR-ed, all others
// are plain stores.
template <int G>
__device__ __forceinline__ void pack16(const uint32_t (&e)[kSymsPerThread],
                                       const uint32_t (&s)[kSymsPerThread], uint32_t p0,
                                       uint32_t wob)
{
    uint32_t hi = 0u, lo = 0u;
    uint32_t wa = imad(p0 >> 5, kc[kFour], wob);  // the word being filled
    uint32_t nbe = p0 & 31u;                      // its bits before this lane, - 32 per word out
    uint32_t shared = nbe != 0;
#pragma unroll
    for (int k = 0; k < kSymsPerThread; ++k) {
        const uint32_t x = e[k];
        hi = __funnelshift_l(lo, hi, x);  // (hi:lo) <<= len
        lo = __funnelshift_l(x, lo, x);   //   ... | code
        if ((k + 1) % G == 0 || k == kSymsPerThread - 1) {
            const uint32_t nb = nbe + s[k];        // pending bits, < 64
            const uint32_t f = nb >> 5;            // a whole word is ready
            put_word(f, shared, wa, __funnelshift_r(lo, hi, nb));  // shift by nb - 32
            wa = imad(f, kc[kFour], wa);
            nbe = imad(f, kc[kMinus32], nbe);
            shared &= f ^ 1u;
        }
    }
    const uint32_t rest = (nbe + s[kSymsPerThread - 1]) & 31u;
    put_word(rest, 1u, wa, __funnelshift_lc(0u, lo, 32 - rest));  // lo << (32 - rest)
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

// Shared per-unit setup of the encoders below.
struct UnitState {
    uint64_t base;   // first symbol of the unit
    uint64_t gbit;   // stream bit of the next step's first symbol
    uint32_t carry;  // bits of the partial word before the step, high-aligned
    uint32_t lead;   // distance from the step start to the next chunk start
    uint64_t next_chunk;  // index of that chunk
    uint4 nxt;       // this lane's 16 input bytes of the coming step
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
    st.nxt = make_uint4(0, 0, 0, 0);
    if (st.base + (uint64_t)lane * kSymsPerThread + kSymsPerThread <= J.n)
        st.nxt = ld_stream16(J.in + st.base + lane * kSymsPerThread);
    return st;
}

// This lane's 16 input bytes of the step starting at symbol sb (m of them
// real, the rest zero), and the load of the next step's bytes.
__device__ __forceinline__ int step_input(const Job &J, UnitState &st, int step, uint64_t sb,
                                          int lane, uint32_t (&w)[4])
{
    const uint64_t i0 = sb + (uint64_t)lane * kSymsPerThread;
    const int m = i0 >= J.n ? 0 : (J.n - i0 >= kSymsPerThread ? kSymsPerThread : (int)(J.n - i0));
    w[0] = st.nxt.x;
    w[1] = st.nxt.y;
    w[2] = st.nxt.z;
    w[3] = st.nxt.w;
    if (step + 1 < kStepsPerUnit && i0 + kStepSyms + kSymsPerThread <= J.n)
        st.nxt = ld_stream16(J.in + i0 + kStepSyms);  // one step ahead
    if (m < kSymsPerThread) {
        w[0] = w[1] = w[2] = w[3] = 0u;
#pragma unroll
        for (int k = 0; k < kSymsPerThread; ++k)
            if (k < m)
                w[k >> 2] |= (uint32_t)J.in[i0 + k] << (8 * (k & 3));
    }
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
// lane's symbols (a chunk starts at a multiple of cs, itself a multiple of
// 16, so only at a lane's first symbol).
__device__ __forceinline__ void step_chunks(const Job &J, const UnitState &st, uint64_t sb,
                                            int lane, uint32_t pos)
{
    if (!J.table_fits)
        return;
    const uint32_t d = (uint32_t)lane * kSymsPerThread;
    uint64_t *offs = reinterpret_cast<uint64_t *>(J.out + kHeaderBytes);
    if (J.cs >= (uint32_t)kStepSyms) {  // at most one start per step
        stg64_if(d == st.lead && sb + d < J.n, offs + st.next_chunk, st.gbit + pos);
    } else if (d >= st.lead && (d - st.lead) % J.cs == 0 && sb + d < J.n) {
        offs[(sb + d) / J.cs] = st.gbit + pos;
    }
}

__device__ __forceinline__ void step_advance(const Job &J, UnitState &st, uint32_t step_bits)
{
    st.gbit += step_bits;
    if (st.lead >= (uint32_t)kStepSyms) {
        st.lead -= kStepSyms;
    } else if (J.cs >= (uint32_t)kStepSyms) {
        st.lead = J.cs - (kStepSyms - st.lead);
        ++st.next_chunk;
    } else {
        st.lead = (J.cs - (kStepSyms - st.lead) % J.cs) % J.cs;
    }
}

// Whole words of the step out (coalesced); the partial last word is carried
// into the next step, or left to the next unit's seam at the unit end.
__device__ __forceinline__ bool step_output(const Job &J, UnitState &st, uint64_t sb,
                                            uint32_t step_bits, const uint32_t *wob, int lane)
{
    uint32_t *pay = reinterpret_cast<uint32_t *>(J.out + J.pay0);
    const uint32_t r = (uint32_t)(st.gbit & 31);
    const uint32_t nw = (r + step_bits + 31) >> 5;
    const bool last = sb + kStepSyms >= J.n;
    const uint32_t tail = (r + step_bits) & 31u;
    const uint32_t nwrite = (last || tail == 0) ? nw : nw - 1;
    const uint64_t wbase = st.gbit >> 5;
    bool overflow = false;
    if (wbase + nwrite <= J.cap_words) {
        // warp-uniform trip count; reading past nwrite stays inside the buffer
        for (uint32_t j0 = 0; j0 < nwrite; j0 += 32) {
            const uint32_t j = j0 + lane;
            stg_if(j < nwrite, pay + wbase + j, wob[j]);
        }
    } else {
        for (uint32_t j = lane; j < nwrite; j += 32) {
            if (wbase + j < J.cap_words)
                pay[wbase + j] = wob[j];
            else
                overflow = true;
        }
    }
    st.carry = tail ? wob[nw - 1] : 0u;
    return overflow;
}

// One 512-symbol step of the fast encoder (codes of at most 24 bits, G =
// floor(32 / longest)).  kInner: the step and the next one lie inside the
// input, the unit is not the last one and its words fit the output, so the
// step needs none of the bound checks.
template <int G, bool kInner>
__device__ __forceinline__ bool fast_step(const Job &J, UnitState &st, int step, int lane,
                                          uint32_t tcol_s, uint32_t wob_s, uint32_t *wob)
{
    const uint64_t sb = st.base + (uint64_t)step * kStepSyms;
    uint32_t w[4];
    int m = kSymsPerThread;
    if (kInner) {
        w[0] = st.nxt.x;
        w[1] = st.nxt.y;
        w[2] = st.nxt.z;
        w[3] = st.nxt.w;
        if (step + 1 < kStepsPerUnit)
            st.nxt = ld_stream16(J.in + sb + kStepSyms + lane * kSymsPerThread);
    } else {
        m = step_input(J, st, step, sb, lane, w);
    }

    // table entries of this lane's symbols and their running bit counts
    uint32_t e[kSymsPerThread], s[kSymsPerThread];
    uint32_t bits = 0;
#pragma unroll
    for (int k = 0; k < kSymsPerThread; ++k) {
        e[k] = tbl_at(imad(byte_of(w, k), kc[k128], tcol_s));
        if (!kInner && k >= m)
            e[k] = 0u;
        bits += e[k] & 31u;
        s[k] = bits;
    }
    uint32_t pos, step_bits;
    scan_bits(bits, lane, pos, step_bits);
    const uint32_t p0 = (uint32_t)(st.gbit & 31) + pos, pend = p0 + bits;

    // words that will be OR-ed start at zero: word 0 holds the carried bits,
    // and each lane clears the word it ends in when that word is shared with
    // the lanes after it
    sts_if(lane == 0, wob_s, st.carry);
    sts_if((pend & 31u) && (pend >> 5), imad(pend >> 5, kc[kFour], wob_s), 0u);
    __syncwarp();
    step_chunks(J, st, sb, lane, pos);
    pack16<G>(e, s, p0, wob_s);
    __syncwarp();
    bool overflow = false;
    if (kInner) {
        // whole words out; the partial last word is carried
        uint32_t *pay = reinterpret_cast<uint32_t *>(J.out + J.pay0);
        const uint32_t r = (uint32_t)(st.gbit & 31);
        const uint32_t tail = (r + step_bits) & 31u;
        const uint32_t nwrite = (r + step_bits) >> 5;
        const uint64_t wbase = st.gbit >> 5;
        for (uint32_t j0 = 0; j0 < nwrite; j0 += 32) {
            const uint32_t j = j0 + lane;
            stg_if(j < nwrite, pay + wbase + j, wob[j]);
        }
        st.carry = tail ? wob[nwrite] : 0u;
    } else {
        overflow = step_output(J, st, sb, step_bits, wob, lane);
    }
    __syncwarp();
    step_advance(J, st, step_bits);
    return overflow;
}

// Encode unit u of job J with the calling warp, codes of at most 24 bits.
// wob is the warp's buffer of kWarpObuf words, tbl the CTA's table.
// Returns true if a payload word fell outside the output capacity.
template <int G>
__device__ __forceinline__ bool encode_unit_fast(const Job &J, uint64_t u, const uint32_t *tbl,
                                                 uint32_t *wob)
{
    const int lane = threadIdx.x & 31;
    const uint32_t tcol_s = smem_u32(tbl + lane), wob_s = smem_u32(wob);
    UnitState st = unit_start(J, u, tbl, true, lane);
    const bool inner = st.base + kUnitSymbols < J.n && (J.unit_off[u + 1] >> 5) < J.cap_words;
    bool overflow = false;
    if (inner) {  // warp-uniform
        for (int step = 0; step < kStepsPerUnit; ++step)
            fast_step<G, true>(J, st, step, lane, tcol_s, wob_s, wob);
    } else {
        for (int step = 0; step < kStepsPerUnit; ++step) {
            if (st.base + (uint64_t)step * kStepSyms >= J.n)
                break;  // warp-uniform
            overflow |= fast_step<G, false>(J, st, step, lane, tcol_s, wob_s, wob);
        }
    }
    return overflow;
}

// The same for codes of up to 32 bits: split code / length tables and a
// 64-bit accumulator (rare: only very skewed inputs have codes this long).
__device__ __forceinline__ bool encode_unit_long(const Job &J, uint64_t u, const uint32_t *tbl,
                                              uint32_t *wob)
{
    const int lane = threadIdx.x & 31;
    bool overflow = false;
    UnitState st = unit_start(J, u, tbl, false, lane);
    for (int step = 0; step < kStepsPerUnit; ++step) {
        const uint64_t sb = st.base + (uint64_t)step * kStepSyms;
        if (sb >= J.n)
            break;  // warp-uniform
        uint32_t w[4];
        const int m = step_input(J, st, step, sb, lane, w);
        uint32_t e[kSymsPerThread], l2[kSymsPerThread];
        uint32_t bits = 0;
        const int col = lane & 15;
#pragma unroll
        for (int k = 0; k < kSymsPerThread; ++k) {
            const uint32_t b = byte_of(w, k);
            e[k] = k < m ? tbl[(b << 4) | col] : 0u;
            l2[k] = k < m ? tbl[256 * 16 + ((b << 4) | col)] : 0u;
            bits += l2[k];
        }
        uint32_t pos, step_bits;
        scan_bits(bits, lane, pos, step_bits);
        const uint32_t r = (uint32_t)(st.gbit & 31);
        const uint32_t nw = (r + step_bits + 31) >> 5;
        for (uint32_t j = lane; j < nw; j += 32)
            wob[j] = j == 0 ? st.carry : 0u;  // word 0 starts with the carried bits
        __syncwarp();
        step_chunks(J, st, sb, lane, pos);
        if (m > 0) {
            uint32_t wi = (r + pos) >> 5, nb = (r + pos) & 31u;
            uint64_t acc = 0;
#pragma unroll
            for (int k = 0; k < kSymsPerThread; ++k) {
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
        overflow |= step_output(J, st, sb, step_bits, wob, lane);
        __syncwarp();
        step_advance(J, st, step_bits);
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
