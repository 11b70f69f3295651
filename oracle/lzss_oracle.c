/*
 * lzss_oracle.c -- plain, slow CPU oracle of LZSS Method 1 and Method 2.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline / reference arm may load this file.  It shares no
 * code, header, table or constant generator with the CUDA library, and the
 * library never calls it.
 *
 * What it computes (paper: "Parallel Data Compression Techniques",
 * Section III-B, LZSS):
 *   - Method 1 codes the data against a sliding window of the W most recent
 *     bits: where the next bits repeat bits of the window for at least a
 *     minimum length, a flag 1, the offset of the repeat and its length are
 *     written; otherwise a flag 0 and the next `block` bits as they are.
 *     The window starts either from a fixed dictionary (counting numbers)
 *     or from the first W bits of the data, stored uncompressed.
 *                                          oracle_lzss_encode / _decode
 *   - Method 2 cuts the data into equal segments, codes each one on its
 *     own, and packs the segments' lengths and codes together in order.
 *                              oracle_lzss_segmented_compress / _decompress
 *
 * Readings of points the paper leaves open (the paper counts window and
 * match lengths in bits, "1024/24/12/8" = window 1024 bits, longest match 24
 * bits, shortest 12 bits, literal block 8 bits):
 *   Z1 bits: data bytes are read most significant bit first.
 *   Z2 parameters: W a power of two in [2, 65536], 1 <= Lmin <= Lmax <= 32,
 *      1 <= B <= 32, dictionary mode D = 1 or 2.
 *   Z3 initial window: D = 1 (counting numbers): the W bits before the
 *      segment are the bytes 0, 1, 2, ... (byte k has value k mod 256), MSB
 *      first.  D = 2 (the first W bits of the file): the first min(W, 8m)
 *      bits of an m-byte segment are written as they are, coding starts after
 *      them and no match reaches before the segment.
 *   Z4 search: at bit p with r bits left, a match is a distance d (1 <= d
 *      <= W, and d <= p when D = 2) and a length l (Lmin <= l <= min(Lmax,
 *      r)) with bit p - d + i equal to bit p + i for every i < l; the source
 *      may run into the bits being coded (positions >= p are the segment's
 *      own bits).  The longest match is used; among equally long ones, the
 *      smallest distance.
 *   Z5 tokens: a match is the bit 1, d - 1 in log2(W) bits, then l - Lmin in
 *      ceil(log2(Lmax - Lmin + 1)) bits (none when Lmax = Lmin), each MSB
 *      first.  Otherwise the bit 0 and the next min(B, r) bits.
 *   Z6 Method 2 container (integers little-endian): [0,8) n; [8,16) segment
 *      bytes S; [16,20) W; [20,24) Lmin; [24,28) Lmax; [28,32) B; [32,36) D;
 *      [36,40) zero; [40,48) count = ceil(n / S); then count u32 bit lengths
 *      of the segments' codes; then the codes, segment i's bits packed MSB
 *      first into bytes from a 16-byte boundary (the first one after the
 *      header and table), zero padded to the next 16-byte boundary.
 *   Z7 decoding validation: the header and table must be consistent (the
 *      container exactly long enough, parameters as in Z2), every distance
 *      within the window, every length within the segment, and a segment's
 *      tokens must end exactly at its recorded bit length.
 *
 * Parity: pinned (hand-worked token streams, an independent brute-force
 * check of every match, round trips, container layout; see
 * tests/test_oracle_lzss.py).
 */
#include "huff_oracle.h"

#include <stdlib.h>
#include <string.h>

static void put_u32le(uint8_t *p, uint32_t v)
{
    for (int k = 0; k < 4; ++k)
        p[k] = (uint8_t)(v >> (8 * k));
}
static void put_u64le(uint8_t *p, uint64_t v)
{
    for (int k = 0; k < 8; ++k)
        p[k] = (uint8_t)(v >> (8 * k));
}
static uint32_t get_u32le(const uint8_t *p)
{
    uint32_t v = 0;
    for (int k = 0; k < 4; ++k)
        v |= (uint32_t)p[k] << (8 * k);
    return v;
}
static uint64_t get_u64le(const uint8_t *p)
{
    uint64_t v = 0;
    for (int k = 0; k < 8; ++k)
        v |= (uint64_t)p[k] << (8 * k);
    return v;
}

/* ---- parameters --------------------------------------------------------- */
static int log2_exact(uint32_t w)
{
    int k = 0;
    while ((1u << k) < w)
        ++k;
    return (1u << k) == w ? k : -1;
}
static int ceil_log2(uint32_t v)
{
    int k = 0;
    while ((1ull << k) < v)
        ++k;
    return k;
}

int oracle_lzss_params_ok(const oracle_lzss_params *P)
{
    return P && P->window >= 2 && P->window <= 65536 && log2_exact(P->window) > 0 &&
           P->min_len >= 1 && P->min_len <= P->max_len && P->max_len <= 32 && P->block >= 1 &&
           P->block <= 32 && (P->dict == 1 || P->dict == 2);
}

/* bits of the offset and length fields */
static int off_bits(const oracle_lzss_params *P) { return log2_exact(P->window); }
static int len_bits(const oracle_lzss_params *P) { return ceil_log2(P->max_len - P->min_len + 1); }

uint64_t oracle_lzss_max_bits(uint64_t m, const oracle_lzss_params *P)
{
    /* every token codes at least min(B, Lmin) bits, except the last literal */
    const uint64_t bits = 8 * m;
    const uint32_t step = P->block < P->min_len ? P->block : P->min_len;
    const uint64_t tok_ref = 1 + (uint64_t)off_bits(P) + (uint64_t)len_bits(P);
    const uint64_t tok_lit = 1 + (uint64_t)P->block;
    const uint64_t tok = tok_ref > tok_lit ? tok_ref : tok_lit;
    return (bits / step + 2) * tok + P->window;
}

/* ---- bit access ----------------------------------------------------------- */
/* bit i of the data, most significant bit of each byte first (Z1) */
static int data_bit(const uint8_t *x, uint64_t i) { return (x[i >> 3] >> (7 - (i & 7))) & 1; }
/* bit j of the counting-numbers dictionary (Z3, D = 1) */
static int dict_bit(uint64_t j) { return (int)((((j >> 3) & 255) >> (7 - (j & 7))) & 1); }

/* bit q of the segment, where q < 0 reads the dictionary before it */
static int seg_bit(const uint8_t *x, int64_t q, uint32_t W)
{
    return q >= 0 ? data_bit(x, (uint64_t)q) : dict_bit((uint64_t)(q + (int64_t)W));
}

typedef struct {
    uint8_t *buf;
    uint64_t cap_bits;
    uint64_t pos;
    int over;
} bitw;

static void put_bits(bitw *w, uint32_t v, int nbits)
{
    for (int k = nbits - 1; k >= 0; --k) {
        if (w->pos >= w->cap_bits) {
            w->over = 1;
            return;
        }
        if ((w->pos & 7) == 0)
            w->buf[w->pos >> 3] = 0; /* a new byte starts clear */
        if ((v >> k) & 1)
            w->buf[w->pos >> 3] |= (uint8_t)(0x80u >> (w->pos & 7));
        ++w->pos;
    }
}

/* ---- Method 1: one segment ------------------------------------------------ */
int oracle_lzss_encode(const uint8_t *x, uint64_t m, const oracle_lzss_params *P, uint8_t *out,
                       uint64_t cap_bytes, uint64_t *bits_out)
{
    if (!oracle_lzss_params_ok(P) || (m && !x) || !bits_out)
        return ORACLE_ERR_INVALID_ARG;
    const uint64_t nbits = 8 * m;
    const uint32_t W = P->window;
    bitw w = {out, 8 * cap_bytes, 0, 0};
    uint64_t p = 0;
    if (P->dict == 2) { /* Z3: the first W bits as they are */
        const uint64_t raw = nbits < W ? nbits : W;
        for (; p < raw; ++p)
            put_bits(&w, (uint32_t)data_bit(x, p), 1);
    }
    while (p < nbits) {
        const uint64_t r = nbits - p;
        const uint64_t maxlen = r < P->max_len ? r : P->max_len;
        uint64_t best_len = 0, best_d = 0;
        if (maxlen >= P->min_len) {
            for (uint64_t d = 1; d <= W; ++d) { /* Z4: every distance, in order */
                if (P->dict == 2 && d > p)
                    break;
                uint64_t l = 0;
                while (l < maxlen &&
                       seg_bit(x, (int64_t)p - (int64_t)d + (int64_t)l, W) ==
                           seg_bit(x, (int64_t)(p + l), W))
                    ++l;
                if (l > best_len) { /* strictly longer: ties keep the smaller d */
                    best_len = l;
                    best_d = d;
                }
            }
        }
        if (best_len >= P->min_len) { /* Z5: a reference */
            put_bits(&w, 1u, 1);
            put_bits(&w, (uint32_t)(best_d - 1), off_bits(P));
            put_bits(&w, (uint32_t)(best_len - P->min_len), len_bits(P));
            p += best_len;
        } else { /* Z5: a literal */
            const uint64_t k = r < P->block ? r : P->block;
            put_bits(&w, 0u, 1);
            for (uint64_t i = 0; i < k; ++i)
                put_bits(&w, (uint32_t)data_bit(x, p + i), 1);
            p += k;
        }
    }
    *bits_out = w.pos;
    return w.over ? ORACLE_ERR_CAPACITY : ORACLE_OK;
}

typedef struct {
    const uint8_t *buf;
    uint64_t nbits;
    uint64_t pos;
} bitr;

static int get_bits(bitr *r, int nbits, uint32_t *v)
{
    uint32_t a = 0;
    for (int k = 0; k < nbits; ++k) {
        if (r->pos >= r->nbits)
            return 0;
        a = (a << 1) | (uint32_t)data_bit(r->buf, r->pos++);
    }
    *v = a;
    return 1;
}

static void set_bit(uint8_t *y, uint64_t i, int b)
{
    if (b)
        y[i >> 3] |= (uint8_t)(0x80u >> (i & 7));
    else
        y[i >> 3] &= (uint8_t)~(0x80u >> (i & 7));
}

int oracle_lzss_decode(const uint8_t *code, uint64_t code_bits, const oracle_lzss_params *P,
                       uint8_t *y, uint64_t m)
{
    if (!oracle_lzss_params_ok(P) || (m && !y))
        return ORACLE_ERR_INVALID_ARG;
    const uint64_t nbits = 8 * m;
    const uint32_t W = P->window;
    bitr r = {code, code_bits, 0};
    uint64_t p = 0;
    uint32_t v;
    if (m)
        memset(y, 0, m);
    if (P->dict == 2) {
        const uint64_t raw = nbits < W ? nbits : W;
        for (; p < raw; ++p) {
            if (!get_bits(&r, 1, &v))
                return ORACLE_ERR_CORRUPT;
            set_bit(y, p, (int)v);
        }
    }
    while (p < nbits) {
        uint32_t flag;
        if (!get_bits(&r, 1, &flag))
            return ORACLE_ERR_CORRUPT;
        const uint64_t rem = nbits - p;
        if (flag) {
            uint32_t dm1, lm;
            if (!get_bits(&r, off_bits(P), &dm1) || !get_bits(&r, len_bits(P), &lm))
                return ORACLE_ERR_CORRUPT;
            const uint64_t d = (uint64_t)dm1 + 1, l = (uint64_t)lm + P->min_len;
            if (l > P->max_len || l > rem || (P->dict == 2 && d > p))
                return ORACLE_ERR_CORRUPT;
            for (uint64_t i = 0; i < l; ++i) { /* bit by bit: the source may overlap */
                const int64_t q = (int64_t)(p + i) - (int64_t)d;
                set_bit(y, p + i, q >= 0 ? data_bit(y, (uint64_t)q) : dict_bit((uint64_t)(q + W)));
            }
            p += l;
        } else {
            const uint64_t k = rem < P->block ? rem : P->block;
            for (uint64_t i = 0; i < k; ++i) {
                if (!get_bits(&r, 1, &v))
                    return ORACLE_ERR_CORRUPT;
                set_bit(y, p + i, (int)v);
            }
            p += k;
        }
    }
    return r.pos == code_bits ? ORACLE_OK : ORACLE_ERR_CORRUPT;
}

/* ---- Method 2: the segmented container ------------------------------------ */
#define LZ_HEAD 48u

static uint64_t al16(uint64_t v) { return (v + 15) & ~(uint64_t)15; }

uint64_t oracle_lzss_segmented_max_size(uint64_t n, uint64_t seg, const oracle_lzss_params *P)
{
    if (!oracle_lzss_params_ok(P) || seg == 0)
        return 0;
    const uint64_t count = n ? (n + seg - 1) / seg : 0;
    uint64_t total = al16(LZ_HEAD + 4 * count);
    for (uint64_t i = 0; i < count; ++i) {
        const uint64_t m = i + 1 < count ? seg : n - i * seg;
        total += al16((oracle_lzss_max_bits(m, P) + 7) / 8);
    }
    return total;
}

int oracle_lzss_segmented_compress(const uint8_t *x, uint64_t n, uint64_t seg,
                                   const oracle_lzss_params *P, uint8_t *out, uint64_t cap,
                                   uint64_t *out_bytes)
{
    if (!oracle_lzss_params_ok(P) || seg == 0 || seg > 0xffffffffull / 8 || (n && !x) ||
        !out_bytes)
        return ORACLE_ERR_INVALID_ARG;
    const uint64_t count = n ? (n + seg - 1) / seg : 0;
    uint64_t pos = al16(LZ_HEAD + 4 * count);
    *out_bytes = 0;
    if (cap < pos)
        return ORACLE_ERR_CAPACITY;
    memset(out, 0, pos);
    put_u64le(out, n);
    put_u64le(out + 8, seg);
    put_u32le(out + 16, P->window);
    put_u32le(out + 20, P->min_len);
    put_u32le(out + 24, P->max_len);
    put_u32le(out + 28, P->block);
    put_u32le(out + 32, P->dict);
    put_u64le(out + 40, count);
    for (uint64_t i = 0; i < count; ++i) {
        const uint64_t m = i + 1 < count ? seg : n - i * seg;
        const uint64_t room = cap - pos;
        uint64_t bits = 0;
        const int st = oracle_lzss_encode(x + i * seg, m, P, out + pos, room, &bits);
        if (st != ORACLE_OK)
            return st;
        put_u32le(out + LZ_HEAD + 4 * i, (uint32_t)bits);
        const uint64_t used = al16((bits + 7) / 8);
        if (used > room)
            return ORACLE_ERR_CAPACITY;
        memset(out + pos + (bits + 7) / 8, 0, used - (bits + 7) / 8);
        pos += used;
    }
    *out_bytes = pos;
    return ORACLE_OK;
}

int oracle_lzss_segmented_decompress(const uint8_t *c, uint64_t bytes, uint8_t *out, uint64_t cap,
                                     uint64_t *n_out)
{
    if (!c || !n_out)
        return ORACLE_ERR_INVALID_ARG;
    *n_out = 0;
    if (bytes < LZ_HEAD)
        return ORACLE_ERR_CORRUPT;
    oracle_lzss_params P;
    const uint64_t n = get_u64le(c), seg = get_u64le(c + 8);
    P.window = get_u32le(c + 16);
    P.min_len = get_u32le(c + 20);
    P.max_len = get_u32le(c + 24);
    P.block = get_u32le(c + 28);
    P.dict = get_u32le(c + 32);
    const uint64_t count = get_u64le(c + 40);
    if (!oracle_lzss_params_ok(&P) || get_u32le(c + 36) != 0 || seg == 0 ||
        seg > 0xffffffffull / 8 || count != (n ? (n + seg - 1) / seg : 0) ||
        count > (bytes - LZ_HEAD) / 4)
        return ORACLE_ERR_CORRUPT;
    uint64_t pos = al16(LZ_HEAD + 4 * count);
    for (uint64_t i = 0; i < count; ++i)
        pos += al16(((uint64_t)get_u32le(c + LZ_HEAD + 4 * i) + 7) / 8);
    if (pos != bytes)
        return ORACLE_ERR_CORRUPT;
    *n_out = n;
    if (n > cap)
        return ORACLE_ERR_CAPACITY;
    pos = al16(LZ_HEAD + 4 * count);
    for (uint64_t i = 0; i < count; ++i) {
        const uint64_t m = i + 1 < count ? seg : n - i * seg;
        const uint64_t bits = get_u32le(c + LZ_HEAD + 4 * i);
        const int st = oracle_lzss_decode(c + pos, bits, &P, out + i * seg, m);
        if (st != ORACLE_OK)
            return st;
        pos += al16((bits + 7) / 8);
    }
    return ORACLE_OK;
}
