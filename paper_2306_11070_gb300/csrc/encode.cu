// Encoder: the coding step of the paper's Huffman Method 1 (Section III-A)
// over Method 2's segments, which become chunks of `cs` symbols with stored
// bit offsets.
//
// Design (one pass over the input, HBM-bound: n bytes read + payload
// written):
//  - The bit offset of every 16 KiB unit is known before this kernel starts
//    (offsets.cu: unit histograms or unit counts, then a scan), so no warp
//    ever waits on another.  Each warp encodes whole units by itself in 32
//    steps of 512 symbols; the loop has no CTA barrier at all.
//  - A step: every lane loads its 16 bytes (one coalesced 16-byte load,
//    issued one step ahead), looks up the 16 table entries and keeps them in
//    registers, a warp scan of the code-length sums gives every lane its bit
//    position, the lanes pack their codes into the warp's word-aligned buffer
//    in shared memory, and the warp writes the whole words with coalesced
//    stores.  The partial last word is carried in a register into the next
//    step.
//  - Code table in shared memory, replicated per lane ([byte][lane]), so
//    the 32 lookups of a warp never collide in a bank.  Entry =
//    (code << (32 - len)) | len for codes up to 24 bits: the funnel shifts
//    take the length from the entry's low 5 bits, so appending a code is two
//    SHF instructions, and the emit check runs once per floor(32 / longest)
//    codes.  Longer codes (up to 32 bits) use split code / length tables and
//    a 64-bit accumulator.
//  - The word a unit shares with the unit before it is completed by the later
//    unit: it re-codes the last <= 31 bits of its predecessor from the 32
//    input bytes before it, so no warp waits for another's output and the
//    payload needs no clearing pass.
#include "huff_internal.cuh"

namespace huff {
namespace {

constexpr int kEncBlock = 256;
constexpr int kEncWarps = kEncBlock / 32;
constexpr int kSymsPerThread = 16;
constexpr int kStepSyms = 32 * kSymsPerThread;          // 512 per warp step
constexpr int kStepsPerUnit = kUnitSymbols / kStepSyms;  // 32
constexpr int kTblWords = 256 * 32;                      // 32 KiB
constexpr int kWarpObuf = kStepSyms + 8;                 // 32-bit codes + alignment
constexpr int kEncSmemBytes = (kTblWords + kEncWarps * kWarpObuf) * 4;
constexpr int kFastMaxLen = 24;

struct EncodeArgs {
    const uint8_t *in;
    uint64_t n;
    const huff_codebook_t *cb;
    const unsigned long long *unit_off;  // exclusive bit prefix per unit, total at [units]
    uint32_t cs;
    uint64_t units;
    uint8_t *out;
    uint64_t out_cap;
    unsigned long long *out_bytes;
    int32_t *status;
};

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

__global__ void __launch_bounds__(kEncBlock, 3) k_encode(EncodeArgs a)
{
    extern __shared__ uint4 smem_raw[];
    uint32_t *tbl = reinterpret_cast<uint32_t *>(smem_raw);  // [256][32] or 2 x [256][16]
    uint32_t *wob = tbl + kTblWords + (threadIdx.x >> 5) * kWarpObuf;  // this warp's buffer

    if (chain_failed(a.status))
        return;
    const int tid = threadIdx.x, lane = tid & 31;
    const uint32_t max_len = a.cb->max_len;
    const bool fast = max_len <= (uint32_t)kFastMaxLen;
    // codes per emit check in the fast path: floor(32 / longest), as a template
    const uint32_t gq = max_len ? 32u / max_len : 16u;
    const int group = gq >= 16 ? 16 : gq >= 8 ? 8 : gq >= 4 ? 4 : gq >= 3 ? 3 : gq >= 2 ? 2 : 1;
    const uint64_t chunks = a.n ? ceil_div_u64(a.n, a.cs) : 0;
    const uint64_t pay0 = kHeaderBytes + 8 * chunks;  // payload byte offset
    const bool table_fits = pay0 <= a.out_cap;
    const uint64_t cap_words = table_fits ? (a.out_cap - pay0) / 4 : 0;
    uint32_t *pay = reinterpret_cast<uint32_t *>(a.out + pay0);

    if (blockIdx.x == 0) {
        if (a.out_cap >= kHeaderBytes) {
            a.out[tid] = a.cb->len[tid];
            if (tid == 0) {
                *reinterpret_cast<uint64_t *>(a.out + 256) = a.n;
                *reinterpret_cast<uint32_t *>(a.out + 264) = a.cs;
                *reinterpret_cast<uint32_t *>(a.out + 268) = max_len;
            }
        }
        if (tid == 0) {
            const uint64_t total = a.units ? a.unit_off[a.units] : 0;
            *a.out_bytes = pay0 + 4 * ((total + 31) >> 5);
            if (!table_fits)
                set_status(a.status, HUFF_ERR_CAPACITY);
        }
    }
    if (fast) {
        for (int i = tid; i < kTblWords; i += kEncBlock) {
            const int b = i >> 5;
            const uint32_t L = a.cb->len[b];
            tbl[i] = L ? (a.cb->code[b] << (32 - L)) | L : 0u;
        }
    } else {
        for (int i = tid; i < 256 * 16; i += kEncBlock) {
            const int b = i >> 4;
            tbl[i] = a.cb->code[b];
            tbl[256 * 16 + i] = a.cb->len[b];
        }
    }
    __syncthreads();  // the only CTA barrier: the table is ready

    const uint32_t *tcol = tbl + lane;
    const uint64_t nwarps = (uint64_t)gridDim.x * kEncWarps;
    bool overflow = false;
    for (uint64_t u = (uint64_t)blockIdx.x * kEncWarps + (tid >> 5); u < a.units; u += nwarps) {
        const uint64_t base = u * kUnitSymbols;
        uint64_t G = a.unit_off[u];
        uint32_t carry = (base > 0 && (G & 31)) ? seam_word(a.in, base, (uint32_t)(G & 31), tbl,
                                                            fast, lane)
                                                 : 0u;
        // distance from the step start to the next chunk start (0 if it is one)
        const uint32_t umod = (uint32_t)(base % a.cs);
        uint32_t lead = umod ? a.cs - umod : 0u;
        uint4 nxt = make_uint4(0, 0, 0, 0);
        if (base + (uint64_t)lane * kSymsPerThread + kSymsPerThread <= a.n)
            nxt = ld_stream16(a.in + base + lane * kSymsPerThread);
        for (int step = 0; step < kStepsPerUnit; ++step) {
            const uint64_t sb = base + (uint64_t)step * kStepSyms;
            if (sb >= a.n)
                break;  // warp-uniform
            const uint64_t i0 = sb + (uint64_t)lane * kSymsPerThread;
            const int m =
                i0 >= a.n ? 0 : (a.n - i0 >= kSymsPerThread ? kSymsPerThread : (int)(a.n - i0));
            uint32_t w[4] = {nxt.x, nxt.y, nxt.z, nxt.w};
            if (step + 1 < kStepsPerUnit && i0 + kStepSyms + kSymsPerThread <= a.n)
                nxt = ld_stream16(a.in + i0 + kStepSyms);  // one step ahead
            if (m < kSymsPerThread) {
                w[0] = w[1] = w[2] = w[3] = 0u;
#pragma unroll
                for (int k = 0; k < kSymsPerThread; ++k)
                    if (k < m)
                        w[k >> 2] |= (uint32_t)a.in[i0 + k] << (8 * (k & 3));
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
            if (m > 0 && table_fits) {
                const uint32_t d = (uint32_t)lane * kSymsPerThread;
                const bool starts = a.cs >= (uint32_t)kStepSyms
                                        ? d == lead
                                        : (d >= lead && (d - lead) % a.cs == 0);
                if (starts)
                    *reinterpret_cast<uint64_t *>(a.out + kHeaderBytes + 8 * (i0 / a.cs)) = G + pos;
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
            const bool last = sb + kStepSyms >= a.n;
            const uint32_t tail = (r + step_bits) & 31u;
            const uint32_t nwrite = (last || tail == 0) ? nw : nw - 1;
            const uint64_t wbase = G >> 5;
            for (uint32_t j = lane; j < nwrite; j += 32) {
                const uint64_t gw = wbase + j;
                if (gw < cap_words)
                    pay[gw] = wob[j];
                else
                    overflow = true;
            }
            carry = tail ? wob[nw - 1] : 0u;
            __syncwarp();
            G += step_bits;
            // the next step starts kStepSyms later
            lead = lead >= (uint32_t)kStepSyms ? lead - kStepSyms
                                               : (a.cs - (kStepSyms - lead) % a.cs) % a.cs;
        }
    }
    if (overflow)
        set_status(a.status, HUFF_ERR_CAPACITY);
}

}  // namespace

uint64_t encode_workspace_bytes(uint64_t n)
{
    const uint64_t units = (n + kUnitSymbols - 1) / kUnitSymbols;
    return ((4 * units + 255) & ~255ull) + 8 * (units + 1);
}

cudaError_t launch_encode(const uint8_t *d_in, uint64_t n, const huff_codebook_t *d_cb, uint32_t cs,
                          uint8_t *d_out, uint64_t out_cap, unsigned long long *d_out_bytes,
                          void *d_ws, const uint16_t *d_unit_hist, int32_t *d_status,
                          cudaStream_t s)
{
    static int per_sm = 0;
    cudaError_t err;
    if (per_sm == 0) {
        err = cudaFuncSetAttribute(k_encode, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   kEncSmemBytes);
        if (err != cudaSuccess)
            return err;
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_encode, kEncBlock,
                                                            kEncSmemBytes);
        if (err != cudaSuccess)
            return err;
        if (per_sm < 1)
            per_sm = 1;
    }
    const uint64_t units = (n + kUnitSymbols - 1) / kUnitSymbols;
    uint8_t *ws = static_cast<uint8_t *>(d_ws);
    uint32_t *unit_bits = reinterpret_cast<uint32_t *>(ws);
    unsigned long long *unit_off =
        reinterpret_cast<unsigned long long *>(ws + ((4 * units + 255) & ~255ull));
    err = launch_unit_offsets(d_in, n, d_unit_hist, d_cb, unit_bits, unit_off, d_status, s);
    if (err != cudaSuccess)
        return err;
    EncodeArgs a;
    a.in = d_in;
    a.n = n;
    a.cb = d_cb;
    a.unit_off = unit_off;
    a.cs = cs;
    a.units = units;
    a.out = d_out;
    a.out_cap = out_cap;
    a.out_bytes = d_out_bytes;
    a.status = d_status;
    uint64_t grid = (uint64_t)device_sm_count() * per_sm;
    const uint64_t want = (units + kEncWarps - 1) / kEncWarps;
    if (grid > want)
        grid = want;
    if (grid < 1)
        grid = 1;
    k_encode<<<(unsigned)grid, kEncBlock, kEncSmemBytes, s>>>(a);
    return cudaGetLastError();
}

}  // namespace huff
