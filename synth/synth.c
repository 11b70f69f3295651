/*
 * Seeded synthetic inputs shared by the CPU oracle tests, the GPU parity
 * tests and the benchmark.  This file holds no Huffman arithmetic: it only
 * draws bytes, sizes and arrival times.
 *
 * Every stream comes from splitmix64 (Steele, Lea and Flood, "Fast
 * splittable pseudorandom number generators", OOPSLA 2014), so the inputs are
 * reproducible from a seed without depending on any library's RNG.
 *
 * The paper's Huffman corpus (a ~45 MB concatenation of English books,
 * Section III-A) is not available, so gen_text() produces text of the same
 * scale and a text-like symbol distribution: words from a random vocabulary
 * with Zipf frequencies, spaces, punctuation and line breaks.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static inline uint64_t sm64(uint64_t *state)
{
    uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* uniform double in [0, 1) with 53 random bits */
static inline double u01(uint64_t *state)
{
    return (double)(sm64(state) >> 11) * (1.0 / 9007199254740992.0);
}

/* uniform integer in [0, m) by multiply-shift of the top 32 bits */
static inline uint32_t below(uint64_t *state, uint32_t m)
{
    return (uint32_t)(((sm64(state) >> 32) * (uint64_t)m) >> 32);
}

/* Cumulative Zipf(s) table over ranks 1..v, normalised to end at 1. */
static double *zipf_cdf(uint32_t v, double s)
{
    double *cdf = (double *)malloc(sizeof(double) * v);
    if (!cdf)
        return NULL;
    double acc = 0.0;
    for (uint32_t k = 0; k < v; ++k) {
        acc += pow((double)(k + 1), -s);
        cdf[k] = acc;
    }
    for (uint32_t k = 0; k < v; ++k)
        cdf[k] /= acc;
    cdf[v - 1] = 1.0;
    return cdf;
}

/* smallest rank index k with u < cdf[k] */
static inline uint32_t zipf_draw(const double *cdf, uint32_t v, double u)
{
    uint32_t lo = 0, hi = v - 1;
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if (u < cdf[mid])
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

/* Guide table for the inverse-CDF search: guide[g] = smallest k with
 * cdf[k] > g / G, so the draw scans forward from guide[floor(u * G)].  Same
 * result as the plain search, a few comparisons per draw. */
enum { GUIDE = 1 << 16 };

static uint32_t *zipf_guide(const double *cdf, uint32_t v)
{
    uint32_t *g = (uint32_t *)malloc(sizeof(uint32_t) * (GUIDE + 1));
    if (!g)
        return NULL;
    uint32_t k = 0;
    for (uint32_t i = 0; i <= GUIDE; ++i) {
        double lo = (double)i / GUIDE;
        while (k < v - 1 && !(lo < cdf[k]))
            ++k;
        g[i] = k;
    }
    return g;
}

static inline uint32_t zipf_draw_guided(const double *cdf, const uint32_t *g, uint32_t v,
                                        double u)
{
    uint32_t k = g[(uint32_t)(u * GUIDE)];
    while (k < v - 1 && !(u < cdf[k]))
        ++k;
    return k;
}

uint64_t synth_splitmix64(uint64_t state) { return sm64(&state); }

/* Bytes i.i.d. Zipf(s) over 96 consecutive codes starting at the space
 * (rank k = 1..96 -> byte 31 + k). */
int synth_zipf_ascii(uint8_t *out, uint64_t n, uint64_t seed, double s)
{
    double *cdf = zipf_cdf(96, s);
    if (!cdf)
        return -1;
    uint64_t st = seed;
    for (uint64_t i = 0; i < n; ++i)
        out[i] = (uint8_t)(32 + zipf_draw(cdf, 96, u01(&st)));
    free(cdf);
    return 0;
}

/* Text: a vocabulary of `vocab` random lowercase words (length geometric
 * with p = 0.3 on {1, 2, ...}, capped at 12), word choice Zipf(1.0) by
 * vocabulary index, 5% of words followed by one of ".,;:!?", then a newline
 * when the line has reached 80 characters and a space otherwise.  The stream
 * is cut at exactly n bytes. */
int synth_text(uint8_t *out, uint64_t n, uint64_t seed)
{
    enum { VOCAB = 50000, MAXW = 12 };
    static const char punct[6] = {'.', ',', ';', ':', '!', '?'};
    uint64_t st = seed;
    uint8_t *words = (uint8_t *)malloc((size_t)VOCAB * MAXW);
    uint8_t *wlen = (uint8_t *)malloc(VOCAB);
    double *cdf = zipf_cdf(VOCAB, 1.0);
    uint32_t *guide = cdf ? zipf_guide(cdf, VOCAB) : NULL;
    if (!words || !wlen || !cdf || !guide) {
        free(words);
        free(wlen);
        free(cdf);
        free(guide);
        return -1;
    }
    for (uint32_t w = 0; w < VOCAB; ++w) {
        uint32_t len = 1;
        while (len < MAXW && !(u01(&st) < 0.3))
            ++len;
        wlen[w] = (uint8_t)len;
        for (uint32_t j = 0; j < len; ++j)
            words[(size_t)w * MAXW + j] = (uint8_t)('a' + below(&st, 26));
    }
    uint64_t pos = 0;
    uint32_t line = 0;
    while (pos < n) {
        uint32_t w = zipf_draw_guided(cdf, guide, VOCAB, u01(&st));
        for (uint32_t j = 0; j < wlen[w] && pos < n; ++j)
            out[pos++] = words[(size_t)w * MAXW + j];
        line += wlen[w];
        if (u01(&st) < 0.05) {
            uint8_t p = (uint8_t)punct[below(&st, 6)];
            if (pos < n)
                out[pos++] = p;
            line += 1;
        }
        if (pos < n) {
            if (line >= 80) {
                out[pos++] = '\n';
                line = 0;
            } else {
                out[pos++] = ' ';
                line += 1;
            }
        }
    }
    free(words);
    free(wlen);
    free(cdf);
    free(guide);
    return 0;
}

/* Uniform bytes: the low byte of each draw. */
void synth_uniform(uint8_t *out, uint64_t n, uint64_t seed)
{
    uint64_t st = seed;
    for (uint64_t i = 0; i < n; ++i)
        out[i] = (uint8_t)sm64(&st);
}

/* Geometric bytes: the number of trailing zero bits of a draw, capped at
 * 255, so P(k) = 2^-(k+1). */
void synth_geometric(uint8_t *out, uint64_t n, uint64_t seed)
{
    uint64_t st = seed;
    for (uint64_t i = 0; i < n; ++i) {
        uint64_t d = sm64(&st);
        unsigned k = d ? (unsigned)__builtin_ctzll(d) : 64u;
        out[i] = (uint8_t)(k > 255 ? 255 : k);
    }
}

/* Geometric symbol with success probability p over {0..255}: used for small
 * skewed alphabets in tests. */
void synth_geometric_p(uint8_t *out, uint64_t n, uint64_t seed, double p)
{
    uint64_t st = seed;
    for (uint64_t i = 0; i < n; ++i) {
        unsigned k = 0;
        while (k < 255 && !(u01(&st) < p))
            ++k;
        out[i] = (uint8_t)k;
    }
}

/* Log-uniform sizes in [lo, hi]: floor(exp(U(ln lo, ln hi))). */
void synth_log_uniform_sizes(uint64_t *sizes, uint32_t count, uint64_t seed,
                             uint64_t lo, uint64_t hi)
{
    uint64_t st = seed;
    double a = log((double)lo), b = log((double)hi);
    for (uint32_t i = 0; i < count; ++i) {
        uint64_t v = (uint64_t)floor(exp(a + (b - a) * u01(&st)));
        sizes[i] = v < lo ? lo : (v > hi ? hi : v);
    }
}

/* Open-loop Poisson arrival trace: exponential gaps with rate `lambda` per
 * second, an operation bit (0 = compress, 1 = decompress) with probability
 * 1/2 each, and log-uniform sizes in [lo, hi]. */
void synth_poisson_trace(double *t_arrive, uint8_t *op, uint64_t *sizes,
                         uint32_t count, uint64_t seed, double lambda,
                         uint64_t lo, uint64_t hi)
{
    uint64_t st = seed;
    double t = 0.0, a = log((double)lo), b = log((double)hi);
    for (uint32_t i = 0; i < count; ++i) {
        double u = u01(&st);
        t += -log(1.0 - u) / lambda;
        t_arrive[i] = t;
        op[i] = (uint8_t)(sm64(&st) >> 63);
        uint64_t v = (uint64_t)floor(exp(a + (b - a) * u01(&st)));
        sizes[i] = v < lo ? lo : (v > hi ? hi : v);
    }
}

/* Fisher-Yates shuffle of a byte buffer in place. */
void synth_shuffle(uint8_t *buf, uint64_t n, uint64_t seed)
{
    uint64_t st = seed;
    for (uint64_t i = n; i > 1; --i) {
        uint64_t j = (uint64_t)(((unsigned __int128)sm64(&st) * i) >> 64);
        uint8_t t = buf[i - 1];
        buf[i - 1] = buf[j];
        buf[j] = t;
    }
}

/* A stand-in for FPGA configuration bitstreams (the paper's LZSS inputs, not
 * available): long runs of zero bytes (unused frames), copies of a few
 * frame templates with one to three bits flipped (repeated configuration
 * with small differences), and stretches of random bytes.  Record kinds in
 * proportion 55 / 30 / 15 %; zero runs 16 + Exp(mean 500) bytes, templates
 * 32..255 bytes (16 of them, drawn first), random stretches 8 + Exp(mean 64)
 * bytes. */
int synth_bitstream(uint8_t *out, uint64_t n, uint64_t seed)
{
    uint64_t st = seed;
    enum { T = 16 };
    uint8_t *tpl = (uint8_t *)malloc(T * 256);
    uint32_t tlen[T];
    if (!tpl)
        return -1;
    for (int t = 0; t < T; ++t) {
        tlen[t] = 32 + below(&st, 224);
        for (uint32_t i = 0; i < tlen[t]; ++i)
            tpl[t * 256 + i] = (uint8_t)sm64(&st);
    }
    uint64_t i = 0;
    while (i < n) {
        const double r = u01(&st);
        uint64_t len;
        if (r < 0.55) {
            len = 16 + (uint64_t)(-log(1.0 - u01(&st)) * 500.0);
            for (uint64_t k = 0; k < len && i < n; ++k)
                out[i++] = 0;
        } else if (r < 0.85) {
            const uint32_t t = below(&st, T);
            const uint64_t at = i;
            len = tlen[t];
            for (uint64_t k = 0; k < len && i < n; ++k)
                out[i++] = tpl[t * 256 + k];
            const uint32_t flips = 1 + below(&st, 3);
            for (uint32_t f = 0; f < flips; ++f) {
                const uint64_t bit = below(&st, (uint32_t)(8 * len));
                if (at + bit / 8 < n)
                    out[at + bit / 8] ^= (uint8_t)(0x80u >> (bit % 8));
            }
        } else {
            len = 8 + (uint64_t)(-log(1.0 - u01(&st)) * 64.0);
            for (uint64_t k = 0; k < len && i < n; ++k)
                out[i++] = (uint8_t)sm64(&st);
        }
    }
    free(tpl);
    return 0;
}
