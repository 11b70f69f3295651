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
    return (w[k >> 2] >> (8 * (k & 3))) & 0xffu;
}

// Append the 16 codes of one lane (fast table entries, len <= 24) at bit p0
// of the warp's word-aligned buffer.  With G = floor(32 / longest code), G
// codes always fit beside fewer than 32 pending bits in the 64-bit
// accumulator, so the emit check runs once per G codes.  Words are whole and
// owned by this lane except the first emitted one when p0 is not word aligned
// (it holds the end of the previous lane's bits) and the final partial one:
// those two are OR-ed, all others are plain stores.
template <int G>
__device__ __forceinline__ void pack16(const uint32_t (&e)[kSymsPerThread], uint32_t p0,
                                       uint32_t *obuf)
{
    uint32_t wi = p0 >> 5, nb = p0 & 31u, hi = 0u, lo = 0u;
    bool shared = nb != 0;
#pragma unroll
    for (int k = 0; k < kSymsPerThread; ++k) {
        const uint32_t x = e[k];
        hi = __funnelshift_l(lo, hi, x);  // (hi:lo) <<= len
        lo = __funnelshift_l(x, lo, x);   //   ... | code
        nb += x & 31u;
        if ((k + 1) % G == 0 || k == kSymsPerThread - 1) {
            if (nb >= 32) {
                nb -= 32;
                const uint32_t w = __funnelshift_r(lo, hi, nb);
                if (shared)
                    atomicOr(obuf + wi, w);
                else
                    obuf[wi] = w;
                shared = false;
                ++wi;
            }
        }
    }
    if (nb)
        atomicOr(obuf + wi, lo << (32 - nb));
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

// Encode unit u of job J with the calling warp; wob is the warp's buffer of
// kWarpObuf words, tbl the CTA's table.  Returns true if a payload word fell
// outside the output capacity.
__device__ __forceinline__ bool encode_unit(const Job &J, uint64_t u, const uint32_t *tbl, bool fast,
                                           int group, uint32_t *wob)
{
    const int lane = threadIdx.x & 31;
    const uint32_t *tcol = tbl + lane;
    uint32_t *pay = reinterpret_cast<uint32_t *>(J.out + J.pay0);
    bool overflow = false;
    const uint64_t base = u * kUnitSymbols;
    uint64_t G = J.unit_off[u];
    uint32_t carry = (base > 0 && (G & 31)) ? seam_word(J.in, base, (uint32_t)(G & 31), tbl,
                                                        fast, lane)
                                             : 0u;
    // distance from the step start to the next chunk start (0 if it is one)
    const uint32_t umod = (uint32_t)(base % J.cs);
    uint32_t lead = umod ? J.cs - umod : 0u;
    uint4 nxt = make_uint4(0, 0, 0, 0);
    if (base + (uint64_t)lane * kSymsPerThread + kSymsPerThread <= J.n)
        nxt = ld_stream16(J.in + base + lane * kSymsPerThread);
    for (int step = 0; step < kStepsPerUnit; ++step) {
        const uint64_t sb = base + (uint64_t)step * kStepSyms;
        if (sb >= J.n)
            break;  // warp-uniform
        const uint64_t i0 = sb + (uint64_t)lane * kSymsPerThread;
        const int m =
            i0 >= J.n ? 0 : (J.n - i0 >= kSymsPerThread ? kSymsPerThread : (int)(J.n - i0));
        uint32_t w[4] = {nxt.x, nxt.y, nxt.z, nxt.w};
        if (step + 1 < kStepsPerUnit && i0 + kStepSyms + kSymsPerThread <= J.n)
            nxt = ld_stream16(J.in + i0 + kStepSyms);  // one step ahead
        if (m < kSymsPerThread) {
            w[0] = w[1] = w[2] = w[3] = 0u;
#pragma unroll
            for (int k = 0; k < kSymsPerThread; ++k)
                if (k < m)
                    w[k >> 2] |= (uint32_t)J.in[i0 + k] << (8 * (k & 3));
        }

        // table entries of this lane's symbols, and their bit count
        uint32_t e[kSymsPerThread], l2[kSymsPerThread];
        uint32_t bits = 0;
        if (fast) {
            if (m == kSymsPerThread) {
#pragma unroll
                for (int k = 0; k < kSymsPerThread; ++k) {
                    e[k] = tcol[byte_of(w, k) << 5];
                    bits += e[k] & 31u;
                }
            } else {
#pragma unroll
                for (int k = 0; k < kSymsPerThread; ++k) {
                    e[k] = k < m ? tcol[byte_of(w, k) << 5] : 0u;
                    bits += e[k] & 31u;
                }
            }
        } else {
            const int col = lane & 15;
#pragma unroll
            for (int k = 0; k < kSymsPerThread; ++k) {
                const uint32_t b = byte_of(w, k);
                e[k] = k < m ? tbl[(b << 4) | col] : 0u;
                l2[k] = k < m ? tbl[256 * 16 + ((b << 4) | col)] : 0u;
                bits += l2[k];
            }
        }

        // warp scan of the bit counts
        uint32_t incl = bits;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d)
                incl += v;
        }
        const uint32_t pos = incl - bits;
        const uint32_t step_bits = __shfl_sync(0xffffffffu, incl, 31);
        const uint32_t r = (uint32_t)(G & 31);
        const uint32_t nw = (r + step_bits + 31) >> 5;
        for (uint32_t j = lane; j < nw; j += 32)
            wob[j] = j == 0 ? carry : 0u;  // word 0 starts with the carried bits
        __syncwarp();

        // bit offset of every chunk that starts at this lane's first symbol
        if (m > 0 && J.table_fits) {
            const uint32_t d = (uint32_t)lane * kSymsPerThread;
            const bool starts = J.cs >= (uint32_t)kStepSyms
                                    ? d == lead
                                    : (d >= lead && (d - lead) % J.cs == 0);
            if (starts)
                *reinterpret_cast<uint64_t *>(J.out + kHeaderBytes + 8 * (i0 / J.cs)) = G + pos;
        }

        // pack this lane's codes into the warp buffer
        if (m > 0) {
            const uint32_t p0 = r + pos;
            if (fast) {
                switch (group) {
                case 16: pack16<16>(e, p0, wob); break;
                case 8: pack16<8>(e, p0, wob); break;
                case 4: pack16<4>(e, p0, wob); break;
                case 3: pack16<3>(e, p0, wob); break;
                case 2: pack16<2>(e, p0, wob); break;
                default: pack16<1>(e, p0, wob); break;
                }
            } else {
                uint32_t wi = p0 >> 5, nb = p0 & 31u;
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
        }
        __syncwarp();

        // whole words out (coalesced); a partial last word is carried into
        // the next step, or left to the next unit's seam at the unit end
        const bool last = sb + kStepSyms >= J.n;
        const uint32_t tail = (r + step_bits) & 31u;
        const uint32_t nwrite = (last || tail == 0) ? nw : nw - 1;
        const uint64_t wbase = G >> 5;
        for (uint32_t j = lane; j < nwrite; j += 32) {
            const uint64_t gw = wbase + j;
            if (gw < J.cap_words)
                pay[gw] = wob[j];
            else
                overflow = true;
        }
        carry = tail ? wob[nw - 1] : 0u;
        __syncwarp();
        G += step_bits;
        // the next step starts kStepSyms later
        lead = lead >= (uint32_t)kStepSyms ? lead - kStepSyms
                                           : (J.cs - (kStepSyms - lead) % J.cs) % J.cs;
    }
    return overflow;
}

}  // namespace enc
}  // namespace huff
