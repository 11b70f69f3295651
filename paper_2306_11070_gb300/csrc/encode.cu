// Encoder: the coding step of the paper's Huffman Method 1 (Section III-A)
// over Method 2's segments, which become chunks of `cs` symbols with stored
// bit offsets.
//
// Design (one pass over the input, HBM-bound: n bytes read + payload
// written):
//  - The bit offset of every 16 KiB unit is known before this kernel starts
//    (offsets.cu: unit histograms or unit counts, then a scan), so CTAs never
//    wait on each other.  Persistent CTAs of 512 threads take units round
//    robin; the next unit is fetched by a 1-D TMA bulk copy into a second
//    shared-memory stage while the current one is packed.
//  - A unit is packed as two 8192-symbol sub-tiles.  Each thread owns 16
//    consecutive symbols and keeps their table entries in registers: the code
//    lengths are summed once, scanned across the CTA, and the same registers
//    are packed.
//  - Code table in shared memory, replicated per lane ([byte][lane]), so
//    the 32 lookups of a warp never collide in a bank.  Entry =
//    (code << (32 - len)) | len for codes up to 24 bits: the funnel shifts
//    take the length from the entry's low 5 bits, so appending a code is two
//    SHF instructions.  Longer codes (up to 32 bits) use split code / length
//    tables and a 64-bit accumulator.
//  - Words are assembled with shared-memory OR into a buffer aligned to the
//    global 32-bit word grid, then written with coalesced stores.  The word a
//    sub-tile shares with the one before it is completed by the later one: it
//    re-codes the last <= 31 bits of its predecessor from the 32 input bytes
//    before it, so no CTA ever waits for another's output and the payload
//    needs no clearing pass.
#include "huff_internal.cuh"

namespace huff {
namespace {

constexpr int kEncBlock = 512;
constexpr int kEncWarps = kEncBlock / 32;
constexpr int kSymsPerThread = 16;
constexpr int kSubSyms = kEncBlock * kSymsPerThread;  // 8192
constexpr int kSubsPerUnit = kUnitSymbols / kSubSyms; // 2
constexpr int kTblWords = 256 * 32;                   // 32 KiB
constexpr int kObufWords = kSubSyms + 4;              // 32-bit codes + alignment word
constexpr int kStageBytes = kUnitSymbols;             // one unit of input
constexpr int kEncSmemBytes = (kTblWords + kObufWords) * 4 + 2 * kStageBytes;
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

// Thread 0: announce and start the bulk copy of unit u's whole 16-byte pieces.
__device__ __forceinline__ void issue_unit_load(const EncodeArgs &a, uint64_t u, uint8_t *stage,
                                                uint64_t *bar)
{
    const uint64_t base = u * kUnitSymbols;
    const uint64_t left = a.n - base;
    const uint32_t bytes =
        (uint32_t)((left < (uint64_t)kUnitSymbols ? left : (uint64_t)kUnitSymbols) & ~15ull);
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(bar, bytes);
    if (bytes)
        tma_load_1d(stage, a.in + base, bytes, bar);
}

__global__ void __launch_bounds__(kEncBlock, 2) k_encode(EncodeArgs a)
{
    extern __shared__ uint4 smem_raw[];
    uint32_t *tbl = reinterpret_cast<uint32_t *>(smem_raw);  // [256][32] or 2 x [256][16]
    uint32_t *obuf = tbl + kTblWords;
    uint8_t *stages = reinterpret_cast<uint8_t *>(obuf + kObufWords);
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ uint32_t s_warp[kEncWarps];
    __shared__ uint32_t s_sub_bits;

    if (chain_failed(a.status))
        return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t max_len = a.cb->max_len;
    const bool fast = max_len <= (uint32_t)kFastMaxLen;
    const uint64_t chunks = a.n ? ceil_div_u64(a.n, a.cs) : 0;
    const uint64_t pay0 = kHeaderBytes + 8 * chunks;  // payload byte offset
    const bool table_fits = pay0 <= a.out_cap;
    const uint64_t cap_words = table_fits ? (a.out_cap - pay0) / 4 : 0;
    uint32_t *pay = reinterpret_cast<uint32_t *>(a.out + pay0);

    if (blockIdx.x == 0) {
        if (a.out_cap >= kHeaderBytes) {
            if (tid < 256)
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
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
        if (blockIdx.x < a.units)
            issue_unit_load(a, blockIdx.x, stages, &bars[0]);
    }
    __syncthreads();

    uint32_t it = 0;
    for (uint64_t u = blockIdx.x; u < a.units; u += gridDim.x, ++it) {
        const int stage = it & 1;
        const uint8_t *sbuf = stages + stage * kStageBytes;
        const bool ok = mbar_wait(&bars[stage], (it >> 1) & 1);
        if (__syncthreads_or(!ok)) {
            if (tid == 0)
                set_status(a.status, HUFF_ERR_TIMEOUT);
            return;
        }
        // the other stage was last read before the previous unit's end barrier
        const uint64_t un = u + gridDim.x;
        if (tid == 0 && un < a.units)
            issue_unit_load(a, un, stages + (stage ^ 1) * kStageBytes, &bars[stage ^ 1]);

        uint64_t G = a.unit_off[u];
        // distance from the unit start to the next chunk start (0 if it is one)
        const uint32_t umod = (uint32_t)((u * kUnitSymbols) % a.cs);
        uint32_t lead = umod ? a.cs - umod : 0u;
        for (int sub = 0; sub < kSubsPerUnit; ++sub) {
            const uint64_t base = u * kUnitSymbols + (uint64_t)sub * kSubSyms;
            if (base >= a.n)
                break;  // uniform: the unit ends in its first sub-tile
            const uint64_t i0 = base + (uint64_t)tid * kSymsPerThread;
            const int m =
                i0 >= a.n ? 0 : (a.n - i0 >= kSymsPerThread ? kSymsPerThread : (int)(a.n - i0));
            uint32_t w[4] = {0u, 0u, 0u, 0u};
            if (m == kSymsPerThread) {
                const uint4 v = *reinterpret_cast<const uint4 *>(sbuf + sub * kSubSyms +
                                                                  tid * kSymsPerThread);
                w[0] = v.x;
                w[1] = v.y;
                w[2] = v.z;
                w[3] = v.w;
            } else {
#pragma unroll
                for (int k = 0; k < kSymsPerThread; ++k)
                    if (k < m)
                        w[k >> 2] |= (uint32_t)a.in[i0 + k] << (8 * (k & 3));
            }

            // table entries of this thread's symbols, and their bit count
            uint32_t e[kSymsPerThread], l2[kSymsPerThread];
            uint32_t bits = 0;
            if (fast) {
#pragma unroll
                for (int k = 0; k < kSymsPerThread; ++k) {
                    e[k] = k < m ? tbl[(byte_of(w, k) << 5) | lane] : 0u;
                    bits += e[k] & 31u;
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

            // CTA-wide exclusive scan of the bit counts
            uint32_t incl = bits;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t v = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d)
                    incl += v;
            }
            if (lane == 31)
                s_warp[warp] = incl;
            __syncthreads();
            if (warp == 0) {
                const uint32_t v = lane < kEncWarps ? s_warp[lane] : 0u;
                uint32_t x = v;
#pragma unroll
                for (int d = 1; d < kEncWarps; d <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
                    if (lane >= d)
                        x += y;
                }
                if (lane < kEncWarps)
                    s_warp[lane] = x - v;
                if (lane == kEncWarps - 1)
                    s_sub_bits = x;
            }
            __syncthreads();
            const uint32_t pos = s_warp[warp] + incl - bits;
            const uint32_t sub_bits = s_sub_bits;
            const uint32_t r = (uint32_t)(G & 31);
            const uint64_t wbase = G >> 5;
            const uint32_t nw = (r + sub_bits + 31) >> 5;
            for (uint32_t j = tid; j < nw; j += kEncBlock)
                obuf[j] = 0u;
            __syncthreads();

            // bit offset of every chunk that starts at this thread's first symbol
            // (chunk starts are 16-symbol aligned; `lead` is the distance from
            // this sub-tile's base to the next chunk start, 32-bit arithmetic)
            if (m > 0 && table_fits) {
                const uint32_t d = (uint32_t)tid * kSymsPerThread;
                const bool starts = a.cs >= (uint32_t)kSubSyms
                                        ? d == lead
                                        : (d >= lead && (d - lead) % a.cs == 0);
                if (starts)
                    *reinterpret_cast<uint64_t *>(a.out + kHeaderBytes + 8 * (i0 / a.cs)) = G + pos;
            }

            // pack this thread's codes into the word-aligned buffer
            if (m > 0) {
                const uint32_t p0 = r + pos;
                uint32_t wi = p0 >> 5, nb = p0 & 31u;
                if (fast) {
                    uint32_t hi = 0u, lo = 0u;
#pragma unroll
                    for (int k = 0; k < kSymsPerThread; ++k) {
                        const uint32_t x = e[k];
                        hi = __funnelshift_l(lo, hi, x);  // (hi:lo) <<= len
                        lo = __funnelshift_l(x, lo, x);   //   ... | code
                        nb += x & 31u;
                        if (nb >= 32) {
                            nb -= 32;
                            atomicOr(obuf + wi, __funnelshift_r(lo, hi, nb));
                            ++wi;
                        }
                    }
                    if (nb)
                        atomicOr(obuf + wi, lo << (32 - nb));
                } else {
                    uint64_t acc = 0;
#pragma unroll
                    for (int k = 0; k < kSymsPerThread; ++k) {
                        const uint32_t L = l2[k];
                        acc = L ? ((acc << L) | e[k]) : acc;
                        nb += L;
                        if (nb >= 32) {
                            nb -= 32;
                            atomicOr(obuf + wi, (uint32_t)(acc >> nb));
                            ++wi;
                        }
                    }
                    if (nb)
                        atomicOr(obuf + wi, (uint32_t)acc << (32 - nb));
                }
            }

            // the word shared with the previous sub-tile: re-code its last r
            // bits from the 32 input bytes before this one (lane l: base-1-l)
            if (warp == 1 && base > 0 && r != 0) {
                const uint32_t b = a.in[base - 1 - lane];
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
                const uint32_t tail = __reduce_or_sync(0xffffffffu, part);
                if (lane == 0)
                    atomicOr(obuf, tail);
            }
            __syncthreads();

            // coalesced copy-out; a partial last word is left to the next sub-tile
            const bool last = base + kSubSyms >= a.n;
            const uint32_t nwrite = (last || ((r + sub_bits) & 31u) == 0) ? nw : nw - 1;
            bool overflow = false;
            for (uint32_t j = tid; j < nwrite; j += kEncBlock) {
                const uint64_t gw = wbase + j;
                if (gw < cap_words)
                    pay[gw] = obuf[j];
                else
                    overflow = true;
            }
            if (overflow)
                set_status(a.status, HUFF_ERR_CAPACITY);
            G += sub_bits;
            // the next sub-tile starts kSubSyms later
            lead = lead >= (uint32_t)kSubSyms ? lead - kSubSyms
                                              : (a.cs - (kSubSyms - lead) % a.cs) % a.cs;
            __syncthreads();
        }
    }
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
    if (grid > units)
        grid = units;
    if (grid < 1)
        grid = 1;
    k_encode<<<(unsigned)grid, kEncBlock, kEncSmemBytes, s>>>(a);
    return cudaGetLastError();
}

}  // namespace huff
