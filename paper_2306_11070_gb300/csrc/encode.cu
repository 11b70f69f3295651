// Encoder: the coding step of the paper's Huffman Method 1 (Section III-A)
// over Method 2's segments, which become chunks of `cs` symbols with stored
// bit offsets.
//
// Design (one pass over the input, HBM-bound: n bytes read + payload
// written):
//  - Persistent CTAs take 4096-symbol tiles from an atomic ticket, so tiles
//    start in index order and every tile's predecessors are already owned
//    by running CTAs.
//  - Each thread owns 16 consecutive symbols (one 16-byte streaming load)
//    and keeps their table entries in registers: the code lengths are
//    summed once, scanned across the CTA, and the same registers are packed.
//  - The tile's starting bit comes from a single-pass decoupled look-back
//    (Merrill & Garland, 2016) over per-tile flags: a tile publishes its bit
//    count, then sums its predecessors' counts back to the first published
//    inclusive prefix, 32 flags per warp step, with a bounded wait.
//  - Code table in shared memory, replicated per lane ([byte][lane]), so
//    the 32 lookups of a warp never collide in a bank.  Entry =
//    (code << (32 - len)) | len for codes up to 24 bits: the funnel shifts
//    take the length from the entry's low 5 bits, so appending a code is two
//    SHF instructions.  Longer codes (up to 32 bits) use split code / length
//    tables and a 64-bit accumulator.
//  - Words are assembled with shared-memory OR into a tile buffer aligned to
//    the global 32-bit word grid, then written with coalesced stores.  The
//    word a tile shares with its predecessor is completed by the tile itself:
//    it re-codes the last <= 31 bits of the predecessor from its last 32
//    input bytes, so no tile ever waits for another tile's output, and the
//    payload needs no clearing pass.
#include "huff_internal.cuh"

namespace huff {
namespace {

constexpr int kEncBlock = 256;
constexpr int kSymsPerThread = 16;
constexpr int kTileSyms = kEncBlock * kSymsPerThread;  // 4096
constexpr int kTblWords = 256 * 32;                    // 32 KiB
constexpr int kObufWords = kTileSyms + 4;              // 32-bit codes + alignment word
constexpr int kEncSmemBytes = (kTblWords + kObufWords) * 4;
constexpr int kFastMaxLen = 24;

constexpr uint64_t kFlagAgg = 1ull << 62;
constexpr uint64_t kFlagPre = 2ull << 62;
constexpr uint64_t kValMask = (1ull << 62) - 1;

// Workspace: [0,4) ticket, [64, 64 + 8*tiles) look-back flags.
constexpr uint64_t kWsFlagsOffset = 64;

struct EncodeArgs {
    const uint8_t *in;
    uint64_t n;
    const huff_codebook_t *cb;
    uint32_t cs;
    uint32_t tiles;
    uint8_t *out;
    uint64_t out_cap;
    unsigned long long *out_bytes;
    unsigned int *ticket;
    unsigned long long *flags;
    int32_t *status;
};

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v)
{
#pragma unroll
    for (int d = 16; d > 0; d >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, d);
    return v;
}

__device__ __forceinline__ uint32_t byte_of(const uint32_t (&w)[4], int k)
{
    return (w[k >> 2] >> (8 * (k & 3))) & 0xffu;
}

// Look-back by warp 0: returns the exclusive bit prefix of tile t, or
// ~0ull on timeout.
__device__ uint64_t tile_lookback(unsigned long long *flags, uint32_t t, uint32_t tile_bits)
{
    const int lane = threadIdx.x & 31;
    if (t == 0) {
        if (lane == 0)
            st_volatile_u64(flags, kFlagPre | tile_bits);
        return 0;
    }
    if (lane == 0)
        st_volatile_u64(flags + t, kFlagAgg | tile_bits);
    uint64_t excl = 0;
    int64_t j = (int64_t)t - 1;
    uint32_t spins = 0;
    for (;;) {
        const int64_t idx = j - lane;
        uint64_t f = idx >= 0 ? ld_volatile_u64(flags + idx) : kFlagPre;
        while (__any_sync(0xffffffffu, (f >> 62) == 0)) {
            if (++spins > kSpinLimit)
                return ~0ull;
            __nanosleep(32);
            if ((f >> 62) == 0)
                f = ld_volatile_u64(flags + idx);
        }
        const unsigned pre = __ballot_sync(0xffffffffu, (f >> 62) == 2);
        if (pre) {
            const int first = __ffs(pre) - 1;
            excl += warp_sum_u64(lane <= first ? (f & kValMask) : 0);
            break;
        }
        excl += warp_sum_u64(f & kValMask);
        j -= 32;
    }
    if (lane == 0)
        st_volatile_u64(flags + t, kFlagPre | (excl + tile_bits));
    return excl;
}

__global__ void __launch_bounds__(kEncBlock) k_encode(EncodeArgs a)
{
    extern __shared__ uint4 smem_raw[];
    uint32_t *tbl = reinterpret_cast<uint32_t *>(smem_raw);  // [256][32] or 2 x [256][16]
    uint32_t *obuf = tbl + kTblWords;
    __shared__ uint32_t s_tile;
    __shared__ uint32_t s_warp[kEncBlock / 32];
    __shared__ uint32_t s_tile_bits;
    __shared__ unsigned long long s_excl;
    __shared__ int s_abort;

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
            a.out[tid] = a.cb->len[tid];
            if (tid == 0) {
                *reinterpret_cast<uint64_t *>(a.out + 256) = a.n;
                *reinterpret_cast<uint32_t *>(a.out + 264) = a.cs;
                *reinterpret_cast<uint32_t *>(a.out + 268) = max_len;
            }
        }
        if (tid == 0) {
            if (!table_fits)
                set_status(a.status, HUFF_ERR_CAPACITY);
            if (a.tiles == 0)
                *a.out_bytes = kHeaderBytes;
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
    if (tid == 0)
        s_abort = 0;
    __syncthreads();

    for (;;) {
        if (tid == 0)
            s_tile = atomicAdd(a.ticket, 1u);
        __syncthreads();
        const uint32_t t = s_tile;
        if (t >= a.tiles)
            break;
        const uint64_t base = (uint64_t)t * kTileSyms;
        const uint64_t i0 = base + (uint64_t)tid * kSymsPerThread;
        const int m = i0 >= a.n ? 0 : (a.n - i0 >= kSymsPerThread ? kSymsPerThread : (int)(a.n - i0));
        uint32_t w[4] = {0u, 0u, 0u, 0u};
        if (m == kSymsPerThread) {
            const uint4 v = ld_stream16(a.in + i0);
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
            uint32_t v = lane < kEncBlock / 32 ? s_warp[lane] : 0u;
            uint32_t x = v;
#pragma unroll
            for (int d = 1; d < kEncBlock / 32; d <<= 1) {
                const uint32_t u = __shfl_up_sync(0xffffffffu, x, d);
                if (lane >= d)
                    x += u;
            }
            const uint32_t total = __shfl_sync(0xffffffffu, x, kEncBlock / 32 - 1);
            if (lane < kEncBlock / 32)
                s_warp[lane] = x - v;
            const uint64_t excl = tile_lookback(a.flags, t, total);
            if (lane == 0) {
                s_tile_bits = total;
                if (excl == ~0ull) {
                    set_status(a.status, HUFF_ERR_TIMEOUT);
                    s_abort = 1;
                    s_excl = 0;
                } else {
                    s_excl = excl;
                }
            }
        }
        __syncthreads();
        if (s_abort)
            break;
        const uint32_t pos = s_warp[warp] + incl - bits;
        const uint32_t tile_bits = s_tile_bits;
        const uint64_t G = s_excl;
        const uint32_t r = (uint32_t)(G & 31);
        const uint64_t wbase = G >> 5;
        const uint32_t nw = (r + tile_bits + 31) >> 5;
        for (uint32_t j = tid; j < nw; j += kEncBlock)
            obuf[j] = 0u;
        __syncthreads();

        // bit offset of every chunk that starts at this thread's first symbol
        if (m > 0 && (i0 % a.cs) == 0 && table_fits)
            *reinterpret_cast<uint64_t *>(a.out + kHeaderBytes + 8 * (i0 / a.cs)) = G + pos;

        // pack this thread's codes into the word-aligned tile buffer
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

        // the word shared with tile t-1: re-code its last r bits from its last
        // 32 input bytes (lane l takes byte base-1-l)
        if (warp == 1 && t > 0 && r != 0) {
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
            uint32_t s = L;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t v = __shfl_up_sync(0xffffffffu, s, d);
                if (lane >= d)
                    s += v;
            }
            const uint32_t before = s - L;  // bits between this code's end and the tile start
            const uint32_t part = (L && before < r) ? code << (32 - r + before) : 0u;
            const uint32_t tail = __reduce_or_sync(0xffffffffu, part);
            if (lane == 0)
                atomicOr(obuf, tail);
        }
        __syncthreads();

        // coalesced copy-out; a partial last word is left to tile t+1
        const bool last = (t == a.tiles - 1);
        const uint32_t nwrite = (last || ((r + tile_bits) & 31u) == 0) ? nw : nw - 1;
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
        if (last && tid == 0)
            *a.out_bytes = pay0 + 4 * ((G + tile_bits + 31) >> 5);
        __syncthreads();
    }
}

}  // namespace

uint64_t encode_workspace_bytes(uint64_t n)
{
    const uint64_t tiles = (n + kTileSyms - 1) / kTileSyms;
    return kWsFlagsOffset + 8 * tiles;
}

cudaError_t launch_encode(const uint8_t *d_in, uint64_t n, const huff_codebook_t *d_cb, uint32_t cs,
                          uint8_t *d_out, uint64_t out_cap, unsigned long long *d_out_bytes,
                          void *d_ws, int32_t *d_status, cudaStream_t s)
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
    const uint64_t tiles = (n + kTileSyms - 1) / kTileSyms;
    err = cudaMemsetAsync(d_ws, 0, encode_workspace_bytes(n), s);
    if (err != cudaSuccess)
        return err;
    EncodeArgs a;
    a.in = d_in;
    a.n = n;
    a.cb = d_cb;
    a.cs = cs;
    a.tiles = (uint32_t)tiles;
    a.out = d_out;
    a.out_cap = out_cap;
    a.out_bytes = d_out_bytes;
    a.ticket = reinterpret_cast<unsigned int *>(d_ws);
    a.flags = reinterpret_cast<unsigned long long *>(static_cast<uint8_t *>(d_ws) + kWsFlagsOffset);
    a.status = d_status;
    uint64_t grid = (uint64_t)device_sm_count() * per_sm;
    if (grid > tiles)
        grid = tiles;
    if (grid < 1)
        grid = 1;
    k_encode<<<(unsigned)grid, kEncBlock, kEncSmemBytes, s>>>(a);
    return cudaGetLastError();
}

}  // namespace huff
