// LZSS Method 2 on the GPU: the segmented parallel version of the paper's
// LZSS coder (Section III-B).  The data is cut into equal segments, each
// coded on its own against a sliding window of its W most recent bits, and
// the segments' code lengths and codes are packed together in order.
//
// Readings (the paper counts window and match lengths in bits; its example
// configuration "1024/24/12/8" is a 1024-bit window, matches of 12..24 bits
// and 8-bit literal blocks):
//  - bits are read most significant bit of each byte first;
//  - the window starts either from the counting numbers (bytes 0, 1, 2, ...
//    before the segment) or from the segment's first W bits, stored as they
//    are (then no match reaches before the segment);
//  - at each position the longest match of Lmin..min(Lmax, bits left) bits
//    is taken, the smallest distance among equally long ones, and a source
//    may run into the bits being coded; a match is the bit 1, distance - 1
//    in log2(W) bits and length - Lmin in ceil(log2(Lmax - Lmin + 1)) bits,
//    a literal the bit 0 and the next min(B, bits left) bits;
//  - container: a 48-byte header (n, segment bytes, W, Lmin, Lmax, B, the
//    dictionary mode, count), count u32 code lengths in bits, then each
//    segment's code packed MSB first into bytes from a 16-byte boundary,
//    zero padded to the next one.
//
// Compression: one warp per segment.  For each token the 32 lanes search
// the window together: lane j tries distances j + 1, j + 33, j + 65, ...;
// their sources all start at the same bit offset within a word, so each
// candidate costs one window word, a funnel shift, an XOR with the 32
// look-ahead bits (its bits past the longest allowed match forced to 1, so
// the count of leading zeros is already capped) and a count of leading
// zeros; one warp max over (length, -distance) keys picks the token, and a
// match shorter than Lmin then reads as a literal.  For windows of 64 to
// 16384 bits the words come from a per-warp ring in shared memory, filled 32
// words at a time as the position advances and stored twice (at i and
// i + R), so a token's candidates read one straight run of words, no wrap.  Every lane keeps the same
// 64-bit output accumulator and lane 0 stores the completed words into the
// segment's worst-case slot of the workspace; a one-CTA scan then lays out
// the header and length table and a gather moves every code into place.
// Decompression: a one-CTA scan checks the header and table and finds every
// segment's start; then one thread per segment decodes its tokens, copying
// a match's bits from the output it has written (a source that overlaps the
// bits being produced repeats with the match distance as its period).
#include <cstdint>

#include "api_trace.h"
#include "huff_internal.cuh"

namespace huff {
namespace {

constexpr uint32_t kLzHead = 48;
constexpr int kLzWarps = 8;                // compress: segments per CTA
constexpr int kLzBlock = 32 * kLzWarps;
constexpr int kScanBlock = 1024;
constexpr uint32_t kMaxWindow = 65536;
constexpr uint32_t kRingMaxWindow = 16384;  // the shared-memory window ring
// dynamic shared memory of the largest ring (W = 16384: 1024 words, twice, per warp)
constexpr size_t kMaxRingSmem = (size_t)kLzWarps * 2 * 1024 * 4;
constexpr uint64_t kMaxSegment = 1ull << 24;
constexpr int kLzDecThreads = 32;              // decompress: one warp per CTA, a segment per thread
constexpr uint32_t kDecRing = 128;             // output words kept per thread (a power of two)
constexpr uint32_t kDecRingMaxWindow = 2048;   // windows whose words fit the ring with 4 to spare
constexpr uint32_t kLzInCells = 8;             // decompress: 16-byte cells of code staged per thread
constexpr uint32_t kLzInFlight = kLzInCells - 1;  // copies left in flight when a word is read

struct LzParams {
    uint32_t W, lmin, lmax, blk, dict;
    uint32_t ob, lb;  // offset and length field bits
};

__host__ __device__ __forceinline__ int ilog2_exact(uint32_t w)
{
    int k = 0;
    while ((1u << k) < w && k < 31)
        ++k;
    return (1u << k) == w ? k : -1;
}
__host__ __device__ __forceinline__ int ceil_log2(uint32_t v)
{
    int k = 0;
    while ((1ull << k) < v)
        ++k;
    return k;
}
__host__ __device__ __forceinline__ bool params_ok(uint32_t W, uint32_t lmin, uint32_t lmax,
                                                   uint32_t blk, uint32_t dict)
{
    return W >= 2 && W <= kMaxWindow && ilog2_exact(W) > 0 && lmin >= 1 && lmin <= lmax &&
           lmax <= 32 && blk >= 1 && blk <= 32 && (dict == 1 || dict == 2);
}
__host__ __device__ __forceinline__ LzParams make_params(uint32_t W, uint32_t lmin, uint32_t lmax,
                                                         uint32_t blk, uint32_t dict)
{
    LzParams P;
    P.W = W;
    P.lmin = lmin;
    P.lmax = lmax;
    P.blk = blk;
    P.dict = dict;
    P.ob = (uint32_t)ilog2_exact(W);
    P.lb = (uint32_t)ceil_log2(lmax - lmin + 1);
    return P;
}
// upper bound of a segment's code bits: every token but the last literal
// codes at least min(B, Lmin) bits
__host__ __device__ __forceinline__ uint64_t max_bits(uint64_t m, const LzParams &P)
{
    const uint64_t step = P.blk < P.lmin ? P.blk : P.lmin;
    const uint64_t ref = 1 + P.ob + P.lb, lit = 1 + P.blk;
    return (8 * m / step + 2) * (ref > lit ? ref : lit) + P.W;
}
__host__ __device__ __forceinline__ uint64_t al16(uint64_t v) { return (v + 15) & ~15ull; }
// bytes of one segment's worst-case slot in the compression workspace
__host__ __device__ __forceinline__ uint64_t slot_bytes(uint64_t seg, const LzParams &P)
{
    return al16((max_bits(seg, P) + 7) / 8);
}

__device__ __forceinline__ uint32_t bswap32(uint32_t v) { return __byte_perm(v, 0u, 0x0123); }

// word q of the counting-numbers dictionary (bytes 4q .. 4q + 3, MSB first)
__device__ __forceinline__ uint32_t dict_word(uint32_t q)
{
    const uint32_t b = (4 * q) & 255;
    return (b << 24) | (((b + 1) & 255) << 16) | (((b + 2) & 255) << 8) | ((b + 3) & 255);
}

// Word q (bits 32q .. 32q + 31, MSB first) of an m-byte segment, zero past
// its end; the segment starts 16-byte aligned.
__device__ __forceinline__ uint32_t seg_word(const uint8_t *x, uint64_t m, uint64_t q)
{
    const uint64_t b = 4 * q;
    if (b + 4 <= m)
        return bswap32(__ldg(reinterpret_cast<const uint32_t *>(x + b)));
    uint32_t v = 0;
    for (int k = 0; k < 4; ++k)
        v = (v << 8) | (b + k < m ? (uint32_t)x[b + k] : 0u);
    return v;
}

// Word vw of the virtual bit string "window before the segment ++ segment"
// (the W dictionary bits occupy words 0 .. W/32 - 1; only used when W >= 32).
__device__ __forceinline__ uint32_t vword(const uint8_t *x, uint64_t m, uint32_t dwords, uint64_t vw)
{
    return vw < dwords ? dict_word((uint32_t)vw) : seg_word(x, m, vw - dwords);
}

// The 32 bits at bit position v of the virtual string (v may be at any bit)
__device__ __forceinline__ uint32_t vbits(const uint8_t *x, uint64_t m, uint32_t W, uint64_t v)
{
    // windows narrower than a word: handle the dictionary bit by bit
    if (W < 32 && v < W) {
        uint32_t out = 0;
        for (int i = 0; i < 32; ++i) {
            const uint64_t t = v + i;
            uint32_t b;
            if (t < W)
                b = (((uint32_t)(t >> 3) & 255) >> (7 - (t & 7))) & 1;
            else
                b = (seg_word(x, m, (t - W) >> 5) >> (31 - ((t - W) & 31))) & 1;
            out = (out << 1) | b;
        }
        return out;
    }
    const uint32_t dwords = W >= 32 ? W / 32 : 0;
    const uint64_t base = W >= 32 ? 0 : W;  // W < 32: the segment starts at virtual bit W
    const uint64_t u = v - base;
    const uint64_t q = u >> 5;
    const uint32_t sh = (uint32_t)(u & 31);
    const uint32_t a = vword(x, m, dwords, q), b = vword(x, m, dwords, q + 1);
    return sh ? __funnelshift_l(b, a, sh) : a;
}

// Bit accumulator that every lane of a warp keeps in step; lane 0 stores
// each completed 32-bit word (MSB-first bytes) into `out`.
struct WarpBits {
    uint64_t acc;
    uint32_t n;     // pending bits (< 32 between appends)
    uint64_t word;  // next word index
    uint32_t *out;
    __device__ __forceinline__ void put(uint32_t v, uint32_t k, bool leader)
    {
        if (k == 0)
            return;
        acc = (acc << k) | (uint64_t)(v >> (32 - k));  // the top k bits of v
        n += k;
        if (n >= 32) {
            n -= 32;
            if (leader)
                out[word] = bswap32((uint32_t)(acc >> n));
            ++word;
        }
    }
    // the last partial word and zero words up to the slot's 16-byte boundary
    __device__ __forceinline__ void finish(bool leader)
    {
        if (leader) {
            uint64_t w = word;
            if (n)
                out[w++] = bswap32((uint32_t)(acc << (32 - n)));
            while (w & 3)
                out[w++] = 0u;
        }
    }
};

// Ring words per warp (R, a power of two): the window's W/32 words, the
// look-ahead's two and a batch of 32 loaded at once.  Stored twice.
__host__ __device__ __forceinline__ uint32_t ring_words(uint32_t W)
{
    uint32_t r = 64;
    while (r < W / 32 + 36)
        r <<= 1;
    return r;
}
__host__ __device__ __forceinline__ bool ring_ok(const LzParams &P)
{
    return P.W >= 64 && P.W <= kRingMaxWindow;
}

// 2^16 from the constant bank: search_run forms its key by one multiply-add
// on the FMA pipe (a visible power of two would become a shift and an add on
// the ALU pipe, which the candidate loop already fills)
static __constant__ uint32_t kKeyScale = 65536u;

// The best key over this lane's candidates from a straight run of window
// words: w points at the word after the one where candidate 0's source
// begins; candidate k's source begins k words lower.
// key = (capped match length << 16) - 32 k; the caller adds 65535 - lane.
template <int NK>
__device__ __forceinline__ int32_t search_run(const uint32_t *w, uint32_t nk, uint32_t sh, uint32_t X,
                                              uint32_t cap)
{
    int32_t best = INT32_MIN;
    uint32_t hiw = w[0];
    if (NK > 0) {
#pragma unroll
        for (int k = 0; k < NK; ++k) {
            const uint32_t low = w[-(k + 1)];
            const uint32_t src = __funnelshift_l(hiw, low, sh);
            hiw = low;
            const int32_t key = (int32_t)imad((uint32_t)__clz((src ^ X) | cap), kKeyScale,
                                              (uint32_t)(-32 * k));
            best = key > best ? key : best;
        }
    } else {
        for (uint32_t k = 0; k < nk; ++k) {
            const uint32_t low = w[-(int)(k + 1)];
            const uint32_t src = __funnelshift_l(hiw, low, sh);
            hiw = low;
            const int32_t key = (int32_t)imad((uint32_t)__clz((src ^ X) | cap), kKeyScale,
                                              0u - 32u * k);
            best = key > best ? key : best;
        }
    }
    return best;
}

__global__ void __launch_bounds__(kLzBlock)
    k_lzss_compress(const uint8_t *__restrict__ in, uint64_t n, uint64_t seg, LzParams P,
                    uint8_t *__restrict__ slots, uint32_t *__restrict__ bits_out,
                    const int32_t *status)
{
    if (chain_failed(status))
        return;
    extern __shared__ uint32_t lz_ring[];
    const int lane = threadIdx.x & 31;
    const uint64_t count = n ? (n + seg - 1) / seg : 0;
    const uint64_t sbytes = slot_bytes(seg, P);
    const bool use_ring = ring_ok(P);
    const uint32_t R = ring_words(P.W);
    uint32_t *ring = lz_ring + (threadIdx.x >> 5) * 2 * R;  // used only when use_ring
    const uint64_t nwarps = (uint64_t)gridDim.x * kLzWarps;
    for (uint64_t s = (uint64_t)blockIdx.x * kLzWarps + (threadIdx.x >> 5); s < count; s += nwarps) {
        const uint8_t *x = in + s * seg;
        const uint64_t m = s + 1 < count ? seg : n - s * seg;
        const uint64_t nbits = 8 * m;
        WarpBits out;
        out.acc = 0;
        out.n = 0;
        out.word = 0;
        out.out = reinterpret_cast<uint32_t *>(slots + s * sbytes);
        uint64_t p = 0;
        if (P.dict == 2) {  // the first W bits as they are
            const uint64_t raw = nbits < P.W ? nbits : P.W;
            for (uint64_t q = 0; q < raw; q += 32) {
                const uint32_t k = raw - q < 32 ? (uint32_t)(raw - q) : 32u;
                out.put(seg_word(x, m, q >> 5), k, lane == 0);
            }
            p = raw;
        }
        const uint64_t vbase = P.W;  // virtual bit of the segment's bit 0
        const uint32_t dwords = P.W >= 32 ? P.W / 32 : 0;
        const uint32_t nk = P.W >= 32 ? P.W / 32 : 1;  // candidates per lane
        // ring: words [hw - R, hw) of the virtual string are held (twice)
        uint64_t hw = vbase + p >= P.W + 64 ? ((vbase + p - P.W) >> 5) - 2 : 0;
        while (p < nbits) {
            const uint64_t r = nbits - p;
            const uint32_t maxlen = r < P.lmax ? (uint32_t)r : P.lmax;
            uint32_t X;  // the 32 look-ahead bits
            if (use_ring) {
                const uint64_t need = ((vbase + p) >> 5) + 2;
                while (hw < need) {  // warp-uniform: 32 words at a time
                    const uint32_t v = vword(x, m, dwords, hw + lane);
                    const uint32_t i = (uint32_t)(hw + lane) & (R - 1);
                    ring[i] = v;
                    ring[i + R] = v;
                    hw += 32;
                    __syncwarp();
                }
                const uint64_t q = (vbase + p) >> 5;
                X = __funnelshift_l(ring[(uint32_t)(q + 1) & (R - 1)], ring[(uint32_t)q & (R - 1)],
                                    (uint32_t)((vbase + p) & 31));
            } else {
                X = vbits(x, m, P.W, vbase + p);
            }
            uint32_t key = 0;
            if (maxlen >= P.lmin && use_ring && (P.dict == 1 || p >= P.W)) {
                // every distance 1..W is allowed: the ring's straight run
                const uint64_t v0 = vbase + p - (uint64_t)lane - 1;
                const uint32_t *w = ring + ((uint32_t)((v0 >> 5) + 1) & (R - 1)) + R;
                const uint32_t cap = maxlen >= 32 ? 0u : 0x80000000u >> maxlen;
                const int32_t best = nk == 32 ? search_run<32>(w, nk, (uint32_t)(v0 & 31), X, cap)
                                              : search_run<0>(w, nk, (uint32_t)(v0 & 31), X, cap);
                key = __reduce_max_sync(0xffffffffu, (uint32_t)(best + (int32_t)(65535 - lane)));
                if ((key >> 16) < P.lmin)
                    key = 0;
            } else if (maxlen >= P.lmin) {
                // lane's sources: virtual bit v_k = vbase + p - (lane + 1) - 32 k
                const uint64_t v0 = vbase + p - (uint64_t)lane - 1;
                if (P.W >= 32) {
                    const uint32_t sh = (uint32_t)(v0 & 31);
                    uint64_t vw = v0 >> 5;
                    uint32_t hiw = vword(x, m, dwords, vw + 1);
                    for (uint32_t k = 0; k < nk; ++k, --vw) {
                        const uint32_t low = vword(x, m, dwords, vw);
                        const uint32_t src = sh ? __funnelshift_l(hiw, low, sh) : low;
                        hiw = low;
                        const uint32_t d = (uint32_t)lane + 1 + 32 * k;
                        uint32_t len = __clz(src ^ X);
                        len = len < maxlen ? len : maxlen;
                        const bool ok = (P.dict == 1 || d <= p) && len >= P.lmin;
                        const uint32_t kk = (len << 16) | (65535u - (d - 1));
                        key = ok && kk > key ? kk : key;
                    }
                } else if ((uint32_t)lane < P.W) {
                    const uint32_t d = (uint32_t)lane + 1;
                    const uint32_t src = vbits(x, m, P.W, v0);
                    uint32_t len = __clz(src ^ X);
                    len = len < maxlen ? len : maxlen;
                    if ((P.dict == 1 || d <= p) && len >= P.lmin)
                        key = (len << 16) | (65535u - (d - 1));
                }
                key = __reduce_max_sync(0xffffffffu, key);
            }
            if (key) {  // a match: 1, d - 1, l - Lmin
                const uint32_t len = key >> 16, dm1 = 65535u - (key & 0xffffu);
                out.put(1u << 31, 1, lane == 0);
                out.put(dm1 << (32 - P.ob), P.ob, lane == 0);
                out.put(P.lb ? (len - P.lmin) << (32 - P.lb) : 0u, P.lb, lane == 0);
                p += len;
            } else {  // a literal: 0, the next min(B, r) bits
                const uint32_t k = r < P.blk ? (uint32_t)r : P.blk;
                out.put(0u, 1, lane == 0);
                out.put(X, k, lane == 0);
                p += k;
            }
        }
        out.finish(lane == 0);
        if (lane == 0)
            bits_out[s] = (uint32_t)(out.word * 32 + out.n);
    }
}

// Header, length table and segment starts of the container; the size into
// *out_bytes, HUFF_ERR_CAPACITY when it exceeds `cap`.
__global__ void __launch_bounds__(kScanBlock)
    k_lzss_layout(uint64_t n, uint64_t seg, LzParams P, const uint32_t *__restrict__ bits,
                  uint64_t *__restrict__ start, uint8_t *__restrict__ out, uint64_t cap,
                  unsigned long long *out_bytes, int32_t *status)
{
    __shared__ unsigned long long s_part[kScanBlock];
    if (chain_failed(status))
        return;
    const int tid = threadIdx.x;
    const uint64_t count = n ? (n + seg - 1) / seg : 0;
    const uint64_t head = al16(kLzHead + 4 * count);
    const uint64_t per = (count + kScanBlock - 1) / kScanBlock;
    const uint64_t b0 = tid * per, b1 = b0 + per < count ? b0 + per : count;
    unsigned long long own = 0;
    for (uint64_t i = b0; i < b1; ++i)
        own += al16((bits[i] + 7) / 8);
    s_part[tid] = own;
    __syncthreads();
    unsigned long long before = 0;
    for (int t = 0; t < tid; ++t)
        before += s_part[t];
    for (uint64_t i = b0; i < b1; ++i) {
        start[i] = head + before;
        before += al16((bits[i] + 7) / 8);
    }
    __syncthreads();
    unsigned long long total = head;
    for (int t = 0; t < kScanBlock; ++t)
        total += s_part[t];
    if (tid == 0) {
        *out_bytes = total;
        if (total > cap)
            set_status(status, HUFF_ERR_CAPACITY);
    }
    if (total > cap)
        return;
    for (uint64_t i = tid; i < head; i += kScanBlock) {  // header, table, padding
        uint8_t v = 0;
        if (i < kLzHead) {
            uint64_t f = 0;
            uint32_t o = (uint32_t)i;
            if (o < 8)
                f = n;
            else if (o < 16)
                f = seg, o -= 8;
            else if (o < 20)
                f = P.W, o -= 16;
            else if (o < 24)
                f = P.lmin, o -= 20;
            else if (o < 28)
                f = P.lmax, o -= 24;
            else if (o < 32)
                f = P.blk, o -= 28;
            else if (o < 36)
                f = P.dict, o -= 32;
            else if (o < 40)
                f = 0, o -= 36;
            else
                f = count, o -= 40;
            v = (uint8_t)(f >> (8 * (o & 7)));
        } else if (i < kLzHead + 4 * count) {
            const uint64_t j = (i - kLzHead) / 4;
            v = (uint8_t)(bits[j] >> (8 * ((i - kLzHead) & 3)));
        }
        out[i] = v;
    }
}

// Move every segment's code from its slot to its place (16-byte copies; the
// slot already holds the zero padding up to its 16-byte boundary).
__global__ void k_lzss_gather(uint64_t n, uint64_t seg, LzParams P, const uint8_t *__restrict__ slots,
                              const uint32_t *__restrict__ bits, const uint64_t *__restrict__ start,
                              uint8_t *__restrict__ out, uint64_t cap, const int32_t *status)
{
    if (chain_failed(status))
        return;
    const uint64_t count = n ? (n + seg - 1) / seg : 0;
    const uint64_t sbytes = slot_bytes(seg, P);
    for (uint64_t s = blockIdx.x; s < count; s += gridDim.x) {
        const uint64_t len = al16((bits[s] + 7) / 8);
        if (start[s] + len > cap)
            continue;
        const uint4 *src = reinterpret_cast<const uint4 *>(slots + s * sbytes);
        uint4 *dst = reinterpret_cast<uint4 *>(out + start[s]);
        for (uint64_t j = threadIdx.x; j < len / 16; j += blockDim.x)
            dst[j] = src[j];
    }
}

// ---------------------------------------------------------------- decompress
// Header and table checks, segment starts (scan), *d_n; statuses as the
// oracle's: CORRUPT for an inconsistent header or table, CAPACITY for n >
// cap.  ok[0] = 1 when the segments may be decoded.
__global__ void __launch_bounds__(kScanBlock)
    k_lzss_dlayout(const uint8_t *__restrict__ c, uint64_t bytes, uint64_t cap,
                   uint64_t *__restrict__ start, uint64_t max_count,
                   unsigned long long *d_n, int32_t *status, uint32_t *ok)
{
    __shared__ unsigned long long s_part[kScanBlock];
    __shared__ int s_bad;
    const int tid = threadIdx.x;
    if (tid == 0) {
        *ok = 0;
        s_bad = 0;
    }
    __syncthreads();
    if (chain_failed(status))
        return;
    if (bytes < kLzHead) {
        if (tid == 0)
            set_status(status, HUFF_ERR_CORRUPT_STREAM);
        return;
    }
    const uint64_t n = *reinterpret_cast<const uint64_t *>(c);
    const uint64_t seg = *reinterpret_cast<const uint64_t *>(c + 8);
    const uint32_t *f = reinterpret_cast<const uint32_t *>(c + 16);
    const uint64_t count = *reinterpret_cast<const uint64_t *>(c + 40);
    const bool hdr_ok = params_ok(f[0], f[1], f[2], f[3], f[4]) && f[5] == 0 && seg >= 16 &&
                        seg % 16 == 0 && seg <= kMaxSegment &&
                        count == (n ? (n + seg - 1) / seg : 0) && count <= (bytes - kLzHead) / 4 &&
                        count <= max_count;
    if (!hdr_ok) {
        if (tid == 0)
            set_status(status, HUFF_ERR_CORRUPT_STREAM);
        return;
    }
    const uint8_t *tab = c + kLzHead;
    const uint64_t head = al16(kLzHead + 4 * count);
    const uint64_t per = (count + kScanBlock - 1) / kScanBlock;
    const uint64_t b0 = tid * per, b1 = b0 + per < count ? b0 + per : count;
    unsigned long long own = 0;
    for (uint64_t i = b0; i < b1; ++i) {
        const uint32_t nb = *reinterpret_cast<const uint32_t *>(tab + 4 * i);
        own += al16(((uint64_t)nb + 7) / 8);
    }
    s_part[tid] = own;
    __syncthreads();
    unsigned long long before = 0, total = head;
    for (int t = 0; t < kScanBlock; ++t) {
        if (t < tid)
            before += s_part[t];
        total += s_part[t];
    }
    for (uint64_t i = b0; i < b1; ++i) {
        start[i] = head + before;
        before += al16(((uint64_t)*reinterpret_cast<const uint32_t *>(tab + 4 * i) + 7) / 8);
    }
    if (tid == 0) {
        if (total != bytes) {
            set_status(status, HUFF_ERR_CORRUPT_STREAM);
            s_bad = 1;
        } else {
            *d_n = n;
            if (n > cap) {
                set_status(status, HUFF_ERR_CAPACITY);
                s_bad = 1;
            }
        }
    }
    __syncthreads();
    if (tid == 0 && !s_bad)
        *ok = 1;
}

// MSB-first bit reader over a segment's code: a 64-bit buffer refilled from
// the code's 32-bit words (the code starts 16-byte aligned and is padded
// with zeros to a 16-byte boundary; words past the padding read as zero).
// The word after the buffer is always loaded one refill ahead, so the
// load's latency is off the token chain.
struct CodeReader {
    const uint32_t *w;
    uint32_t nw;     // words of the padded code
    uint32_t next;   // next word to load
    uint32_t nxt;    // word next - 1, loaded ahead
    uint64_t buf;    // valid bits, left-aligned
    uint32_t have;
    uint32_t nbits;  // the segment's code length (< 2^28: segments are at most 16 MiB)
    uint32_t pos;    // bits consumed
    __device__ __forceinline__ uint32_t load(uint32_t i) const
    {
        return i < nw ? bswap32(__ldg(w + i)) : 0u;
    }
    __device__ __forceinline__ void init(const uint8_t *c, uint64_t code_bits)
    {
        w = reinterpret_cast<const uint32_t *>(c);
        nw = (uint32_t)(al16((code_bits + 7) / 8) / 4);
        buf = ((uint64_t)load(0) << 32) | load(1);
        have = 64;
        nxt = load(2);
        next = 3;
        nbits = (uint32_t)code_bits;
        pos = 0;
    }
    __device__ __forceinline__ uint32_t get(uint32_t k)  // k <= 32 bits, right-aligned
    {
        if (k == 0)
            return 0;
        const uint32_t v = (uint32_t)(buf >> (64 - k));
        buf <<= k;
        have -= k;
        pos += k;
        if (have <= 32) {  // refill: >= 32 valid bits for the next get
            buf |= (uint64_t)nxt << (32 - have);
            have += 32;
            nxt = load(next++);
        }
        return v;
    }
};

// Store output word q (MSB-first bytes) of an m-byte segment output.
__device__ __forceinline__ void store_out_word(uint8_t *y, uint64_t m, uint64_t q, uint32_t w)
{
    const uint64_t b = 4 * q;
    if (b + 4 <= m) {
        reinterpret_cast<uint32_t *>(y)[q] = bswap32(w);
    } else {
        for (int k = 0; k < 4; ++k)
            if (b + k < m)
                y[b + k] = (uint8_t)(w >> (24 - 8 * k));
    }
}

// The bits a thread has produced so far, read back: completed words from
// the output (or, with a ring, from the thread's ring of recent words in
// shared memory), the pending word from its register; positions before the
// segment from the counting-numbers dictionary.  With a ring, completed
// words are written out four at a time with one 16-byte store.
template <bool kRing>
struct OutBits {
    uint8_t *y;      // the segment's output (16-byte aligned)
    uint32_t m;      // its bytes (at most 16 MiB)
    uint32_t W;
    uint32_t *ring;  // kRing: kDecRing words, word q at q mod kDecRing
    uint32_t pend;   // bits of the word being filled, left-aligned
    uint32_t npend;  // their count
    uint32_t pos;    // bits produced (< 2^27)
    __device__ __forceinline__ uint32_t word_at(int32_t q) const  // output word q (may be < 0)
    {
        if (q < 0) {  // the dictionary: virtual word q + W/32 (W >= 32 here)
            return dict_word((uint32_t)(q + (int32_t)(W / 32)));
        }
        if ((uint32_t)q == (pos >> 5))
            return pend;
        if ((uint32_t)q > (pos >> 5))
            return 0u;
        if (kRing)
            return ring[(uint32_t)q & (kDecRing - 1)];
        return bswap32(__ldcg(reinterpret_cast<const uint32_t *>(y) + q));
    }
    // the 32 bits at output bit s (s may be negative: the dictionary)
    __device__ __forceinline__ uint32_t bits_at(int32_t s) const
    {
        if (W < 32 && s < 0) {  // narrow dictionary, bit by bit
            uint32_t out = 0;
            for (int i = 0; i < 32; ++i) {
                const int32_t t = s + i;
                uint32_t b;
                if (t < 0) {
                    const uint32_t j = (uint32_t)(t + (int32_t)W);
                    b = (((uint32_t)(j >> 3) & 255) >> (7 - (j & 7))) & 1;
                } else {
                    b = (word_at(t >> 5) >> (31 - (t & 31))) & 1;
                }
                out = (out << 1) | b;
            }
            return out;
        }
        const int32_t q = s >> 5;  // floor
        const uint32_t sh = (uint32_t)(s & 31);
        const uint32_t a = word_at(q), b = word_at(q + 1);
        return sh ? __funnelshift_l(b, a, sh) : a;
    }
    // append the top k (1..32) bits of v
    __device__ __forceinline__ void put(uint32_t v, uint32_t k)
    {
        v = k < 32 ? v & ~(0xffffffffu >> k) : v;
        const uint64_t acc = ((uint64_t)pend << 32) | ((uint64_t)v << (32 - npend));
        const uint32_t total = npend + k;
        if (total >= 32) {
            complete(pos >> 5, (uint32_t)(acc >> 32));
            pend = (uint32_t)acc;
            npend = total - 32;
        } else {
            pend = (uint32_t)(acc >> 32);
            npend = total;
        }
        pos += k;
    }
    __device__ __forceinline__ void complete(uint32_t q, uint32_t w) const
    {
        if (!kRing) {
            if (4 * q + 4 <= m)
                __stcg(reinterpret_cast<uint32_t *>(y) + q, bswap32(w));
            else
                store_out_word(y, m, q, w);
            return;
        }
        ring[(uint32_t)q & (kDecRing - 1)] = w;
        if ((q & 3) == 3) {  // a whole 16-byte group
            const uint32_t g = q >> 2;
            if (16 * g + 16 <= m) {
                const uint32_t r = (uint32_t)(q - 3) & (kDecRing - 1);
                *reinterpret_cast<uint4 *>(y + 16 * g) =
                    make_uint4(bswap32(ring[r]), bswap32(ring[r + 1]), bswap32(ring[r + 2]),
                               bswap32(ring[r + 3]));
            } else {
                for (uint32_t j = q - 3; j <= q; ++j)
                    store_out_word(y, m, j, ring[(uint32_t)j & (kDecRing - 1)]);
            }
        }
    }
    __device__ __forceinline__ void finish() const
    {
        const uint32_t q = pos >> 5;  // the word being filled
        if (kRing)  // completed words of the last, unfinished group
            for (uint32_t j = q & ~3u; j < q; ++j)
                store_out_word(y, m, j, ring[(uint32_t)j & (kDecRing - 1)]);
        if (npend)
            store_out_word(y, m, q, pend);
    }
};

// The code words of the fast loop below come through a per-thread ring of
// kLzInCells 16-byte cells in shared memory ([cell][thread], 512-byte rows),
// filled by cp.async copies kept ahead of the reader: the 32 lanes of a warp
// refill at different tokens, and a refill that waited on a global load
// would wait on the one another lane issued a token before (the scoreboard
// is the warp's), which left most of the load latency exposed.
__device__ __forceinline__ void lz_cp_async16(uint32_t dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void lz_cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void lz_cp_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

struct CodeRing {
    uint32_t col;      // shared address of this thread's cell in row 0
    uint32_t fetched;  // cells requested so far (cell c holds code words 4c..4c+3)
    uint32_t ncells;   // cells of the segment's code (its 16-byte padded length)
    // request cells until the ring holds the kLzInCells from word w's on
    __device__ __forceinline__ void top_up(const uint32_t *w, uint32_t word)
    {
        while (fetched < (word >> 2) + kLzInCells && fetched < ncells) {
            lz_cp_async16(col + (fetched & (kLzInCells - 1)) * (kLzDecThreads * 16), w + 4 * fetched);
            lz_cp_commit();
            ++fetched;
        }
    }
    // code word `word` right after top_up(w, word): unless the code's last
    // cell has been requested, exactly kLzInFlight cells were requested after
    // word's (one copy group each), so waiting for all but that many to land
    // includes word's; after the last cell every copy is waited for.  A slot
    // is requested again only once the reader has left its cell.
    __device__ __forceinline__ uint32_t word_at(uint32_t word) const
    {
        if (fetched >= ncells)
            lz_cp_wait<0>();
        else
            lz_cp_wait<kLzInFlight>();
        return lds(col + ((word >> 2) & (kLzInCells - 1)) * (kLzDecThreads * 16) + (word & 3u) * 4);
    }
};

// Tokens far from both ends of a segment, for the shared-memory ring
// (windows of 32..2048 bits) with the stored-prefix window and literal blocks
// of at most 31 bits: at least 64 code bits and 32 output bits remain, so no
// bounds check applies, the window never reaches before the output (the
// prefix filled it) and a token is at most 32 bits of the reader's top 32.
// Branch free where the lanes of a warp (each on its own segment) would
// diverge: both the match and the literal are formed and the token
// selects.  False (and the caller's status) only for a length field above
// the longest match.
__device__ __forceinline__ bool decode_fast(CodeReader &rd, OutBits<true> &ob, const LzParams &P,
                                            uint32_t nbits, uint32_t in_col)
{
    CodeRing rg;
    rg.col = in_col;
    rg.fetched = rd.next >> 2;
    rg.ncells = rd.nw >> 2;
    rg.top_up(rd.w, rd.next);
    bool ok = true;
    while (rd.pos + 64 <= rd.nbits && ob.pos + 32 <= nbits) {
        const uint32_t t = (uint32_t)(rd.buf >> 32);  // >= 33 bits are valid
        const uint32_t flag = t >> 31;
        const uint32_t body = t << 1;  // the token after its flag, left-aligned
        const uint32_t d = (body >> (32 - P.ob)) + 1;
        const uint32_t len = (P.lb ? (body << P.ob) >> (32 - P.lb) : 0u) + P.lmin;
        if (flag && len > P.lmax) {
            ok = false;
            break;
        }
        const uint32_t used = flag ? 1u + P.ob + P.lb : 1u + P.blk;
        const uint32_t nout = flag ? len : P.blk;
        // the match's 32 source bits at ob.pos - d (at most W back, so inside
        // the output and the ring; read whether or not the token is a match)
        const uint32_t src = ob.pos - d;
        const uint32_t q = src >> 5, cur = ob.pos >> 5;
        const uint32_t wa = ob.ring[q & (kDecRing - 1)], wb = ob.ring[(q + 1) & (kDecRing - 1)];
        const uint32_t a = q == cur ? ob.pend : wa;
        const uint32_t b = q + 1 == cur ? ob.pend : (q + 1 > cur ? 0u : wb);
        uint32_t v = __funnelshift_l(b, a, src & 31u);
        // a source that runs into the bits being produced repeats with period d
        uint32_t vp = v & ~(0xffffffffu >> (d & 31u));
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            const uint32_t sh = d << i;
            vp |= sh < len ? vp >> (sh & 31u) : 0u;
        }
        v = flag ? (d < len ? vp : v) : body;
        // consume the token: one refill keeps >= 33 bits; the next word
        // comes from the ring (zero past the padded code, as rd.load gives)
        rd.buf <<= used;
        rd.have -= used;
        rd.pos += used;
        if (rd.have <= 32) {
            rd.buf |= (uint64_t)rd.nxt << (32 - rd.have);
            rd.have += 32;
            uint32_t nw = 0u;
            if (rd.next < rd.nw) {
                rg.top_up(rd.w, rd.next);
                nw = bswap32(rg.word_at(rd.next));
            }
            rd.nxt = nw;
            ++rd.next;
        }
        ob.put(v, nout);
    }
    lz_cp_wait<0>();  // no copy in flight into the ring once the loop is left
    return ok;
}

// Decode one segment's tokens; false if the code is corrupt.
template <bool kRing>
__device__ __forceinline__ bool decode_segment(CodeReader &rd, OutBits<kRing> &ob, const LzParams &P,
                                               uint32_t nbits, uint32_t in_col = 0)
{
    if (P.dict == 2) {
        const uint32_t raw = nbits < P.W ? nbits : P.W;
        while (ob.pos < raw) {
            const uint32_t k = raw - ob.pos < 32 ? (uint32_t)(raw - ob.pos) : 32u;
            if (rd.pos + k > rd.nbits)
                return false;
            ob.put(rd.get(k) << (32 - k), k);
        }
    }
    if constexpr (kRing) {
        if (P.dict == 2 && P.blk <= 31 && !decode_fast(rd, ob, P, nbits, in_col))
            return false;
    }
    while (ob.pos < nbits) {
        if (rd.pos >= rd.nbits)
            return false;
        const uint32_t r = nbits - ob.pos;
        if (rd.get(1)) {
            if (rd.pos + P.ob + P.lb > rd.nbits)
                return false;
            const uint32_t d = rd.get(P.ob) + 1;
            const uint32_t len = rd.get(P.lb) + P.lmin;
            if (len > P.lmax || len > r || (P.dict == 2 && d > ob.pos))
                return false;
            uint32_t v = ob.bits_at((int32_t)ob.pos - (int32_t)d);
            if (d < len) {  // the source runs into these bits: period d
                v &= ~(0xffffffffu >> d);
                for (uint32_t sh = d; sh < len; sh <<= 1)
                    v |= v >> sh;
            }
            ob.put(v, len);
        } else {
            const uint32_t k = r < P.blk ? (uint32_t)r : P.blk;
            if (rd.pos + k > rd.nbits)
                return false;
            ob.put(rd.get(k) << (32 - k), k);
        }
    }
    return rd.pos == rd.nbits;
}

// One thread per segment.  Windows of up to kDecRingMaxWindow bits keep the
// thread's recent output words in a shared-memory ring (the matches' source
// words are read there, not back through L2, and output leaves in 16-byte
// stores); wider windows read their sources back from the output.
__global__ void __launch_bounds__(kLzDecThreads) k_lzss_decode(const uint8_t *__restrict__ c,
                                                               const uint64_t *__restrict__ start,
                                                               uint8_t *__restrict__ out,
                                                               int32_t *status, const uint32_t *ok)
{
    // ring of thread t at t * (kDecRing + 1): the odd stride spreads the
    // threads' equal ring positions over the banks
    __shared__ uint32_t rings[kLzDecThreads * (kDecRing + 1)];
    __shared__ __align__(16) uint4 in_ring[kLzInCells * kLzDecThreads];  // [cell][thread]
    if (!*ok || chain_failed(status))
        return;
    const uint32_t in_col = smem_u32(in_ring) + threadIdx.x * 16;
    const uint64_t n = *reinterpret_cast<const uint64_t *>(c);
    const uint64_t seg = *reinterpret_cast<const uint64_t *>(c + 8);
    const uint32_t *f = reinterpret_cast<const uint32_t *>(c + 16);
    const LzParams P = make_params(f[0], f[1], f[2], f[3], f[4]);
    const uint64_t count = *reinterpret_cast<const uint64_t *>(c + 40);
    const bool use_ring = P.W >= 32 && P.W <= kDecRingMaxWindow;
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < count;
         s += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t m = s + 1 < count ? seg : n - s * seg;
        CodeReader rd;
        rd.init(c + start[s], *reinterpret_cast<const uint32_t *>(c + kLzHead + 4 * s));
        bool good;
        if (use_ring) {
            OutBits<true> ob;
            ob.y = out + s * seg;
            ob.m = (uint32_t)m;
            ob.W = P.W;
            ob.ring = rings + threadIdx.x * (kDecRing + 1);
            ob.pend = 0;
            ob.npend = 0;
            ob.pos = 0;
            good = decode_segment(rd, ob, P, (uint32_t)(8 * m), in_col);
            if (good)
                ob.finish();
        } else {
            OutBits<false> ob;
            ob.y = out + s * seg;
            ob.m = (uint32_t)m;
            ob.W = P.W;
            ob.ring = nullptr;
            ob.pend = 0;
            ob.npend = 0;
            ob.pos = 0;
            good = decode_segment(rd, ob, P, (uint32_t)(8 * m));
            if (good)
                ob.finish();
        }
        if (!good)
            set_status(status, HUFF_ERR_CORRUPT_STREAM);
    }
}

__global__ void k_lzss_set(int32_t *status, unsigned long long *p, uint64_t v)
{
    *status = 0;
    if (p)
        *p = v;
}

inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

bool host_params(const huff_lzss_params_t *p, LzParams &P)
{
    if (!p || !params_ok(p->window, p->min_len, p->max_len, p->block, p->dict))
        return false;
    P = make_params(p->window, p->min_len, p->max_len, p->block, p->dict);
    return true;
}

bool seg_ok(uint64_t seg) { return seg >= 16 && seg % 16 == 0 && seg <= kMaxSegment; }

}  // namespace
}  // namespace huff

using namespace huff;

extern "C" {

uint64_t huff_lzss_max_size(uint64_t n, uint64_t segment_bytes, const huff_lzss_params_t *params)
{
    LzParams P;
    if (!host_params(params, P) || !seg_ok(segment_bytes))
        return 0;
    const uint64_t count = n ? (n + segment_bytes - 1) / segment_bytes : 0;
    return al16(kLzHead + 4 * count) + count * slot_bytes(segment_bytes, P);
}

uint64_t huff_lzss_workspace_size(uint64_t n, uint64_t segment_bytes,
                                  const huff_lzss_params_t *params)
{
    LzParams P;
    if (!host_params(params, P) || !seg_ok(segment_bytes))
        return 0;
    const uint64_t count = n ? (n + segment_bytes - 1) / segment_bytes : 0;
    // slots, then the bit lengths (u32) and the starts (u64)
    return count * slot_bytes(segment_bytes, P) + al16(4 * count) + 8 * count + 16;
}

huff_status_t huff_lzss_compress(const uint8_t *d_in, uint64_t n, uint64_t segment_bytes,
                                 const huff_lzss_params_t *params, uint8_t *d_out, uint64_t out_cap,
                                 uint64_t *d_out_bytes, void *d_ws, uint64_t ws_bytes,
                                 int32_t *d_status, huff_stream_t stream)
{
    HUFF_API_RANGE("huff_lzss_compress");
    LzParams P;
    if (!host_params(params, P) || !seg_ok(segment_bytes) || !d_out || !d_out_bytes ||
        !d_status || (n && (!d_in || !aligned16(d_in))) || !aligned16(d_out) ||
        (n && (!d_ws || !aligned16(d_ws))) ||
        ws_bytes < huff_lzss_workspace_size(n, segment_bytes, params))
        return HUFF_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    k_lzss_set<<<1, 1, 0, s>>>(d_status, reinterpret_cast<unsigned long long *>(d_out_bytes), 0);
    const uint64_t count = n ? (n + segment_bytes - 1) / segment_bytes : 0;
    uint8_t *ws = static_cast<uint8_t *>(d_ws);
    uint8_t *slots = ws;
    uint32_t *bits = reinterpret_cast<uint32_t *>(ws + count * slot_bytes(segment_bytes, P));
    uint64_t *start = reinterpret_cast<uint64_t *>(reinterpret_cast<uint8_t *>(bits) + al16(4 * count));
    const int sms = device_sm_count();
    if (sms < 1)
        return HUFF_ERR_CUDA;
    if (count) {
        const size_t smem = ring_ok(P) ? (size_t)kLzWarps * 2 * ring_words(P.W) * 4 : 0;
        static KernelSetup setup;
        int per_sm = 0;
        if (kernel_setup(setup, (const void *)k_lzss_compress, kLzBlock, kMaxRingSmem, &per_sm) !=
            cudaSuccess)
            return HUFF_ERR_CUDA;
        uint64_t grid = (count + kLzWarps - 1) / kLzWarps;
        if (grid > (uint64_t)sms * 64)
            grid = (uint64_t)sms * 64;
        k_lzss_compress<<<(unsigned)grid, kLzBlock, smem, s>>>(d_in, n, segment_bytes, P, slots, bits,
                                                               d_status);
    }
    k_lzss_layout<<<1, kScanBlock, 0, s>>>(n, segment_bytes, P, bits, start, d_out, out_cap,
                                           reinterpret_cast<unsigned long long *>(d_out_bytes),
                                           d_status);
    if (count) {
        const uint64_t grid = count < (uint64_t)sms * 16 ? count : (uint64_t)sms * 16;
        k_lzss_gather<<<(unsigned)grid, 128, 0, s>>>(n, segment_bytes, P, slots, bits, start, d_out,
                                                     out_cap, d_status);
    }
    return cudaGetLastError() == cudaSuccess ? HUFF_OK : HUFF_ERR_CUDA;
}

uint64_t huff_lzss_decompress_workspace_size(uint64_t in_bytes)
{
    const uint64_t max_count = in_bytes > kLzHead ? (in_bytes - kLzHead) / 4 : 0;
    return 16 + 8 * max_count;
}

huff_status_t huff_lzss_decompress(const uint8_t *d_in, uint64_t in_bytes, uint8_t *d_out,
                                   uint64_t out_cap, uint64_t *d_n, void *d_ws, uint64_t ws_bytes,
                                   int32_t *d_status, huff_stream_t stream)
{
    HUFF_API_RANGE("huff_lzss_decompress");
    if (!d_in || !aligned16(d_in) || !d_n || !d_status || (out_cap && !d_out) ||
        (d_out && !aligned16(d_out)) || !d_ws || !aligned16(d_ws) ||
        ws_bytes < huff_lzss_decompress_workspace_size(in_bytes))
        return HUFF_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    k_lzss_set<<<1, 1, 0, s>>>(d_status, reinterpret_cast<unsigned long long *>(d_n), 0);
    const uint64_t max_count = in_bytes > kLzHead ? (in_bytes - kLzHead) / 4 : 0;
    uint32_t *ok = static_cast<uint32_t *>(d_ws);
    uint64_t *start = reinterpret_cast<uint64_t *>(static_cast<uint8_t *>(d_ws) + 16);
    k_lzss_dlayout<<<1, kScanBlock, 0, s>>>(d_in, in_bytes, out_cap, start, max_count,
                                            reinterpret_cast<unsigned long long *>(d_n), d_status,
                                            ok);
    const int sms = device_sm_count();
    if (sms < 1)
        return HUFF_ERR_CUDA;
    // one thread per segment; the count is only known on the device, so
    // bound the grid by the table size
    uint64_t grid = (max_count + kLzDecThreads - 1) / kLzDecThreads;
    if (grid > (uint64_t)sms * 32)
        grid = (uint64_t)sms * 32;
    if (grid < 1)
        grid = 1;
    k_lzss_decode<<<(unsigned)grid, kLzDecThreads, 0, s>>>(d_in, start, d_out, d_status, ok);
    return cudaGetLastError() == cudaSuccess ? HUFF_OK : HUFF_ERR_CUDA;
}

}  // extern "C"
