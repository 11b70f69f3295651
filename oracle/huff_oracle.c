/*
 * huff_oracle.c -- plain, slow CPU oracle of the Huffman hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline / reference arm may load this file.  It shares no
 * code, header, table or constant generator with the CUDA library, and the
 * library never calls it.
 *
 * What it computes (paper: "Parallel Data Compression Techniques",
 * Section III-A, Huffman Method 1 and Method 2):
 *   1. Method 1 counts how often each byte occurs (its "probability of
 *      occurrence").                                        oracle_histogram
 *   2. Method 1 builds an extended weighted binary tree: the two lightest
 *      nodes are replaced by one internal node whose weight is the sum of
 *      theirs, repeated until one root is left.  A leaf's depth is the length
 *      of its code.                                      oracle_code_lengths
 *   3. Codes are assigned canonically from the lengths.
 *                                                     oracle_canonical_codes
 *   4. Encoding concatenates the codes of the input bytes.  Method 2's
 *      segments with ids become fixed-size chunks of `cs` symbols whose
 *      starting bit offsets are recorded, so each chunk can be decoded on
 *      its own and the output reassembled in chunk order.     oracle_encode
 *   5. Decoding ("lossless") reverses 4 chunk by chunk.       oracle_decode
 *   6. Method 3 first applies the block-sorting (Burrows-Wheeler) transform
 *      to every block, and its inverse after decoding.
 *                                                 oracle_bwt / oracle_ibwt
 *      Optionally followed by move-to-front coding per block.
 *                                               oracle_mtf / oracle_imtf
 *
 * Readings of points the paper leaves open:
 *   R1 tie-break: nodes are ordered by (weight, id); leaf id = byte value,
 *      internal ids are 256, 257, ... in creation order.
 *   R2 "replacing two external nodes" is read as the standard step: any two
 *      lowest-(weight, id) nodes, leaves or internal.
 *   R3 empty input: all lengths 0.  Exactly one distinct byte: length 1,
 *      code "0".
 *   R4 a code longer than 32 bits is an error (no length limiting).
 *   R5 canonical order: symbols sorted by (length, byte value); the code
 *      starts at 0 and is shifted left by the length increase before each
 *      assignment, then incremented.
 *   R6 stream: [0,256) lengths u8; [256,264) n u64 LE; [264,268) chunk
 *      symbols u32 LE; [268,272) longest length u32 LE; then ceil(n/cs) u64
 *      LE bit offsets; then the payload as u32 LE words, stream bit j being
 *      bit (31 - j%32) of word j/32 (MSB first), zero padded.
 *   R7 decode validation: see oracle_decode.
 *
 * Parity: pinned (worked examples, Kraft equality, brute-force optimality,
 * Shannon bounds, Fibonacci length boundary, independent offset sums, round
 * trip; see tests/test_oracle_*.py).
 */
#include "huff_oracle.h"

#include <stdlib.h>
#include <string.h>

/* ---- little-endian field access (independent of the host's byte order) */
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

static int chunk_symbols_ok(uint32_t cs)
{
    return cs >= ORACLE_MIN_CHUNK && cs <= ORACLE_MAX_CHUNK && cs % 16 == 0;
}

/* ---- step 1: byte counts ------------------------------------------------ */
void oracle_histogram(const uint8_t *x, uint64_t n, uint64_t hist[256])
{
    memset(hist, 0, 256 * sizeof(uint64_t));
    for (uint64_t i = 0; i < n; ++i)
        hist[x[i]] += 1;
}

/* ---- step 2: the weighted tree, with a binary min-heap on (weight, id) --- */
typedef struct {
    uint64_t w;
    uint32_t id;
} node_t;

static int node_before(node_t a, node_t b)
{
    return a.w < b.w || (a.w == b.w && a.id < b.id);
}

static void heap_push(node_t *h, int *size, node_t v)
{
    int i = (*size)++;
    h[i] = v;
    while (i > 0) {
        int up = (i - 1) / 2;
        if (!node_before(h[i], h[up]))
            break;
        node_t t = h[i];
        h[i] = h[up];
        h[up] = t;
        i = up;
    }
}

static node_t heap_pop(node_t *h, int *size)
{
    node_t top = h[0];
    h[0] = h[--(*size)];
    int i = 0;
    for (;;) {
        int l = 2 * i + 1, r = l + 1, m = i;
        if (l < *size && node_before(h[l], h[m]))
            m = l;
        if (r < *size && node_before(h[r], h[m]))
            m = r;
        if (m == i)
            break;
        node_t t = h[i];
        h[i] = h[m];
        h[m] = t;
        i = m;
    }
    return top;
}

int oracle_code_lengths(const uint64_t hist[256], uint8_t len[256])
{
    node_t heap[512];
    int size = 0, parent[511], leaves = 0, last_leaf = -1;

    memset(len, 0, 256);
    for (int s = 0; s < 256; ++s) {
        parent[s] = -1;
        if (hist[s] > 0) {
            node_t leaf = {hist[s], (uint32_t)s};
            heap_push(heap, &size, leaf);
            ++leaves;
            last_leaf = s;
        }
    }
    if (leaves == 0)
        return ORACLE_OK; /* R3: empty input */
    if (leaves == 1) {
        len[last_leaf] = 1; /* R3: one distinct byte */
        return ORACLE_OK;
    }
    /* R1/R2: replace the two lightest nodes by their sum, until one is left */
    uint32_t next_id = 256;
    while (size > 1) {
        node_t a = heap_pop(heap, &size);
        node_t b = heap_pop(heap, &size);
        node_t inner = {a.w + b.w, next_id++};
        parent[a.id] = (int)inner.id;
        parent[b.id] = (int)inner.id;
        parent[inner.id] = -1;
        heap_push(heap, &size, inner);
    }
    /* code length = depth of the leaf = number of edges up to the root */
    int too_long = 0;
    for (int s = 0; s < 256; ++s) {
        if (hist[s] == 0)
            continue;
        int depth = 0;
        for (int v = s; parent[v] != -1; v = parent[v])
            ++depth;
        if (depth > ORACLE_MAX_CODE_LEN)
            too_long = 1;
        len[s] = (uint8_t)(depth > 255 ? 255 : depth);
    }
    if (too_long) {
        memset(len, 0, 256);
        return ORACLE_ERR_CODE_TOO_LONG; /* R4 */
    }
    return ORACLE_OK;
}

/* ---- step 2', length-limited: package-merge ---------------------------------
 * Not in the paper: an extension of its tree step that keeps every code
 * within `limit` bits (Larmore & Hirschberg, "A fast algorithm for optimal
 * length-restricted Huffman codes", 1990).  Readings:
 *   L1 when the Huffman lengths of step 2 already fit, they are the answer;
 *   L2 otherwise the coin-collector construction: list 1 = the present
 *      symbols sorted by (weight, byte); list i = list 1 merged with the
 *      packages (sums of consecutive pairs) of list i-1, a symbol before a
 *      package of equal weight; the first 2n-2 items of list `limit` are
 *      taken, and each taken package takes its two items of the list below;
 *      a symbol's length is the number of taken items that contain it;
 *   L3 limit outside 1..32 is an invalid argument; more distinct symbols
 *      than 2^limit cannot be coded (CODE_TOO_LONG); one symbol: length 1.
 */
typedef struct {
    uint64_t w;
    int leaf; /* index into the sorted symbols, or -1 for a package */
} item_t;

int oracle_code_lengths_limited(const uint64_t hist[256], uint32_t limit, uint8_t len[256])
{
    uint64_t sw[256];
    int sid[256], n = 0;
    if (limit < 1 || limit > ORACLE_MAX_CODE_LEN)
        return ORACLE_ERR_INVALID_ARG;
    int st = oracle_code_lengths(hist, len);
    if (st == ORACLE_OK) {
        uint32_t mx = 0;
        for (int s = 0; s < 256; ++s)
            if (len[s] > mx)
                mx = len[s];
        if (mx <= limit)
            return ORACLE_OK; /* L1 */
    }
    memset(len, 0, 256);
    /* the present symbols sorted by (weight, byte): insertion sort */
    for (int s = 0; s < 256; ++s) {
        if (!hist[s])
            continue;
        int j = n++;
        while (j > 0 && (sw[j - 1] > hist[s] || (sw[j - 1] == hist[s] && sid[j - 1] > s))) {
            sw[j] = sw[j - 1];
            sid[j] = sid[j - 1];
            --j;
        }
        sw[j] = hist[s];
        sid[j] = s;
    }
    if (limit < 32 && (uint64_t)n > (1ull << limit))
        return ORACLE_ERR_CODE_TOO_LONG; /* L3 */
    /* lists 1..limit; list i has at most 2n - 1 items */
    item_t *lists = (item_t *)malloc(sizeof(item_t) * (size_t)limit * 512);
    int cnt[ORACLE_MAX_CODE_LEN + 1];
    if (!lists)
        return ORACLE_ERR_INVALID_ARG;
    for (int j = 0; j < n; ++j) {
        lists[j].w = sw[j];
        lists[j].leaf = j;
    }
    cnt[1] = n;
    for (uint32_t i = 2; i <= limit; ++i) {
        const item_t *prev = lists + (size_t)(i - 2) * 512;
        item_t *cur = lists + (size_t)(i - 1) * 512;
        const int np = cnt[i - 1] / 2;
        int a = 0, b = 0, k = 0;
        while (a < n || b < np) {
            const uint64_t pw = b < np ? prev[2 * b].w + prev[2 * b + 1].w : 0;
            if (a < n && (b >= np || sw[a] <= pw)) { /* symbol first on a tie */
                cur[k].w = sw[a];
                cur[k].leaf = a;
                ++a;
            } else {
                cur[k].w = pw;
                cur[k].leaf = -1;
                ++b;
            }
            ++k;
        }
        cnt[i] = k;
    }
    /* take the first 2n-2 items of the last list and walk down */
    int take = 2 * n - 2;
    for (uint32_t i = limit; i >= 1 && take > 0; --i) {
        const item_t *cur = lists + (size_t)(i - 1) * 512;
        int packages = 0;
        for (int k = 0; k < take; ++k) {
            if (cur[k].leaf >= 0)
                len[sid[cur[k].leaf]] += 1;
            else
                ++packages;
        }
        take = 2 * packages;
    }
    free(lists);
    if (n == 1)
        len[sid[0]] = 1; /* L3 */
    return ORACLE_OK;
}

/* ---- step 3: canonical codes (R5) ---------------------------------------- */
void oracle_canonical_codes(const uint8_t len[256], uint32_t code[256])
{
    uint64_t next = 0;
    int prev = -1;
    memset(code, 0, 256 * sizeof(uint32_t));
    for (int L = 1; L <= ORACLE_MAX_CODE_LEN; ++L) {
        for (int s = 0; s < 256; ++s) {
            if (len[s] != L)
                continue;
            if (prev < 0)
                next = 0;
            else
                next <<= (L - prev);
            prev = L;
            code[s] = (uint32_t)next;
            next += 1;
        }
    }
}

uint64_t oracle_max_stream_size(uint64_t n, uint32_t cs)
{
    uint64_t chunks = cs ? (n + cs - 1) / cs : 0;
    return ORACLE_HEADER_BYTES + 8 * chunks + 4 * ((n + 3) / 4) + 4;
}

/* ---- step 4: encode ------------------------------------------------------ */
int oracle_chunk_offsets(const uint8_t *x, uint64_t n, uint32_t cs,
                         const uint8_t len[256], uint64_t *off, uint64_t *total_bits)
{
    uint64_t pos = 0;
    if (!chunk_symbols_ok(cs))
        return ORACLE_ERR_INVALID_ARG;
    for (uint64_t i = 0; i < n; ++i) {
        if (i % cs == 0)
            off[i / cs] = pos;
        if (len[x[i]] == 0)
            return ORACLE_ERR_INVALID_ARG; /* byte missing from the codebook */
        pos += len[x[i]];
    }
    *total_bits = pos;
    return ORACLE_OK;
}

int oracle_pack_bits(const uint8_t *x, uint64_t m, const uint8_t len[256],
                     uint32_t *words, uint64_t nwords, uint64_t *bits)
{
    uint32_t code[256];
    uint64_t pos = 0;
    oracle_canonical_codes(len, code);
    memset(words, 0, nwords * sizeof(uint32_t));
    for (uint64_t i = 0; i < m; ++i) {
        int L = len[x[i]];
        if (L == 0)
            return ORACLE_ERR_INVALID_ARG;
        for (int b = L - 1; b >= 0; --b) { /* most significant bit first */
            if ((pos >> 5) >= nwords)
                return ORACLE_ERR_CAPACITY;
            if ((code[x[i]] >> b) & 1u)
                words[pos >> 5] |= 1u << (31 - (pos & 31));
            ++pos;
        }
    }
    *bits = pos;
    return ORACLE_OK;
}

int oracle_encode(const uint8_t *x, uint64_t n, uint32_t cs, const uint8_t len[256],
                  uint8_t *out, uint64_t cap, uint64_t *out_bytes)
{
    uint64_t chunks, total_bits = 0, nwords, need, bits;
    uint32_t max_len = 0;
    int st;

    *out_bytes = 0;
    if (!chunk_symbols_ok(cs))
        return ORACLE_ERR_INVALID_ARG;
    chunks = (n + cs - 1) / cs;
    uint64_t *off = (uint64_t *)malloc(sizeof(uint64_t) * (chunks ? chunks : 1));
    if (!off)
        return ORACLE_ERR_INVALID_ARG;
    st = oracle_chunk_offsets(x, n, cs, len, off, &total_bits);
    if (st != ORACLE_OK) {
        free(off);
        return st;
    }
    nwords = (total_bits + 31) / 32;
    need = ORACLE_HEADER_BYTES + 8 * chunks + 4 * nwords;
    *out_bytes = need;
    if (need > cap) {
        free(off);
        return ORACLE_ERR_CAPACITY;
    }
    for (int s = 0; s < 256; ++s)
        if (len[s] > max_len)
            max_len = len[s];
    memcpy(out, len, 256);
    put_u64le(out + 256, n);
    put_u32le(out + 264, cs);
    put_u32le(out + 268, max_len);
    for (uint64_t c = 0; c < chunks; ++c)
        put_u64le(out + ORACLE_HEADER_BYTES + 8 * c, off[c]);
    free(off);

    uint32_t *words = (uint32_t *)malloc(sizeof(uint32_t) * (nwords ? nwords : 1));
    if (!words)
        return ORACLE_ERR_INVALID_ARG;
    st = oracle_pack_bits(x, n, len, words, nwords, &bits);
    if (st == ORACLE_OK) {
        uint8_t *pay = out + ORACLE_HEADER_BYTES + 8 * chunks;
        for (uint64_t j = 0; j < nwords; ++j)
            put_u32le(pay + 4 * j, words[j]);
    }
    free(words);
    return st;
}

int oracle_compress(const uint8_t *x, uint64_t n, uint32_t cs, uint8_t *out, uint64_t cap,
                    uint64_t *out_bytes)
{
    uint64_t hist[256];
    uint8_t len[256];
    int st;
    *out_bytes = 0;
    oracle_histogram(x, n, hist);
    st = oracle_code_lengths(hist, len);
    if (st != ORACLE_OK)
        return st;
    return oracle_encode(x, n, cs, len, out, cap, out_bytes);
}

/* ---- step 5: decode -------------------------------------------------------
 * Validation (R7), in this order; every failure is "corrupt" except (c):
 *  (a) at least 272 bytes; chunk symbols a multiple of 16 in range; the
 *      offset table fits; every length <= 32 and the largest equals the
 *      header's field; n > 0 needs at least one code; one code must have
 *      length 1; two or more codes must fill the code space exactly
 *      (sum of 2^-len == 1).
 *  (b) *n_out = n.
 *  (c) n larger than the output capacity -> capacity error.
 *  (d) off[0] == 0, offsets non-decreasing and <= payload bits P, where P is
 *      32 * (whole u32 words after the offset table).
 *  (e) chunk c reads only bits below off[c+1] (below P for the last chunk),
 *      every code is found within the longest length, and a chunk that is
 *      not the last one ends exactly at off[c+1].
 */
int oracle_decode(const uint8_t *s, uint64_t bytes, uint8_t *out, uint64_t cap, uint64_t *n_out)
{
    uint8_t len[256];
    uint32_t code[256];
    uint64_t n, chunks;
    uint32_t cs, max_field, max_len = 0, nsym = 0;

    *n_out = 0;
    if (bytes < ORACLE_HEADER_BYTES)
        return ORACLE_ERR_CORRUPT;
    memcpy(len, s, 256);
    n = get_u64le(s + 256);
    cs = get_u32le(s + 264);
    max_field = get_u32le(s + 268);
    if (!chunk_symbols_ok(cs))
        return ORACLE_ERR_CORRUPT;
    chunks = n / cs + (n % cs != 0);
    if (chunks > (bytes - ORACLE_HEADER_BYTES) / 8)
        return ORACLE_ERR_CORRUPT;
    for (int k = 0; k < 256; ++k) {
        if (len[k] > ORACLE_MAX_CODE_LEN)
            return ORACLE_ERR_CORRUPT;
        if (len[k] > max_len)
            max_len = len[k];
        nsym += len[k] > 0;
    }
    if (max_len != max_field)
        return ORACLE_ERR_CORRUPT;
    if (n > 0 && nsym == 0)
        return ORACLE_ERR_CORRUPT;
    if (nsym == 1 && max_len != 1)
        return ORACLE_ERR_CORRUPT;
    if (nsym >= 2) {
        uint64_t kraft = 0; /* sum of 2^(32 - len): 2^32 means sum 2^-len = 1 */
        for (int k = 0; k < 256; ++k)
            if (len[k])
                kraft += (uint64_t)1 << (32 - len[k]);
        if (kraft != ((uint64_t)1 << 32))
            return ORACLE_ERR_CORRUPT;
    }
    *n_out = n;
    if (n > cap)
        return ORACLE_ERR_CAPACITY;

    const uint8_t *offp = s + ORACLE_HEADER_BYTES;
    const uint8_t *pay = offp + 8 * chunks;
    uint64_t pbits = 32 * ((bytes - ORACLE_HEADER_BYTES - 8 * chunks) / 4);
    for (uint64_t c = 0; c < chunks; ++c) {
        uint64_t o = get_u64le(offp + 8 * c);
        if (c == 0 && o != 0)
            return ORACLE_ERR_CORRUPT;
        if (c > 0 && o < get_u64le(offp + 8 * (c - 1)))
            return ORACLE_ERR_CORRUPT;
        if (o > pbits)
            return ORACLE_ERR_CORRUPT;
    }

    /* canonical codes of each length are consecutive integers: decode by
     * the first code and the symbols of each length in byte order */
    uint32_t first[ORACLE_MAX_CODE_LEN + 1], count[ORACLE_MAX_CODE_LEN + 1];
    uint8_t syms[ORACLE_MAX_CODE_LEN + 1][256];
    oracle_canonical_codes(len, code);
    memset(count, 0, sizeof(count));
    memset(first, 0, sizeof(first));
    for (int L = 1; L <= ORACLE_MAX_CODE_LEN; ++L)
        for (int k = 0; k < 256; ++k)
            if (len[k] == L) {
                if (count[L] == 0)
                    first[L] = code[k];
                syms[L][count[L]++] = (uint8_t)k;
            }

    for (uint64_t c = 0; c < chunks; ++c) {
        uint64_t pos = get_u64le(offp + 8 * c);
        uint64_t limit = c + 1 < chunks ? get_u64le(offp + 8 * (c + 1)) : pbits;
        uint64_t base = c * cs;
        uint64_t m = n - base < cs ? n - base : cs;
        for (uint64_t i = 0; i < m; ++i) {
            uint32_t v = 0;
            int L = 0, found = 0;
            while (!found) {
                if (pos >= limit)
                    return ORACLE_ERR_CORRUPT;
                uint32_t word = get_u32le(pay + 4 * (pos >> 5));
                v = (v << 1) | ((word >> (31 - (pos & 31))) & 1u);
                ++pos;
                ++L;
                if (count[L] && v >= first[L] && v - first[L] < count[L]) {
                    out[base + i] = syms[L][v - first[L]];
                    found = 1;
                } else if ((uint32_t)L >= max_len) {
                    return ORACLE_ERR_CORRUPT;
                }
            }
        }
        if (c + 1 < chunks && pos != limit)
            return ORACLE_ERR_CORRUPT;
    }
    return ORACLE_OK;
}

/* ---- Method 3: the block-sorting transform before Huffman coding ---------
 * Method 3 (Section III-A) runs the Burrows-Wheeler transform over each
 * block of the data set and then the parallel Huffman coder of Method 2 over
 * the result.  The paper's one-line description of the transform (an order
 * reversal done by a sort) is garbled; the reading taken is the transform of
 * Burrows and Wheeler (SRC Research Report 124, 1994):
 *   B1 a block is a run of `block` consecutive input bytes (the last block
 *      may be shorter); blocks are transformed independently;
 *   B2 the m cyclic rotations of a block are sorted lexicographically by
 *      unsigned byte value; equal rotations (a periodic block) keep the
 *      order of their starting positions;
 *   B3 the block's output is the last byte of every rotation in sorted
 *      order, and its primary index is the row of the rotation that starts
 *      at the block's first byte.
 * The inverse follows the same report: the last column, sorted stably,
 * gives the first column, and the map from a row to the row of the rotation
 * one byte earlier walks the block backwards from the primary row. */

/* compare the rotations of b[0, m) starting at j and k */
static int rotation_cmp(const uint8_t *b, uint32_t m, uint32_t j, uint32_t k)
{
    for (uint32_t t = 0; t < m; ++t) {
        uint8_t u = b[(uint32_t)(((uint64_t)j + t) % m)];
        uint8_t v = b[(uint32_t)(((uint64_t)k + t) % m)];
        if (u != v)
            return u < v ? -1 : 1;
    }
    return 0;
}

/* stable bottom-up merge sort of the rotation starts idx[0, m) */
static void sort_rotations(const uint8_t *b, uint32_t m, uint32_t *idx, uint32_t *tmp)
{
    for (uint32_t w = 1; w < m; w *= 2) {
        for (uint32_t lo = 0; lo < m; lo += 2 * w) {
            uint32_t mid = lo + w < m ? lo + w : m;
            uint32_t hi = lo + 2 * w < m ? lo + 2 * w : m;
            uint32_t i = lo, j = mid, o = lo;
            while (i < mid && j < hi)
                tmp[o++] = rotation_cmp(b, m, idx[j], idx[i]) < 0 ? idx[j++] : idx[i++];
            while (i < mid)
                tmp[o++] = idx[i++];
            while (j < hi)
                tmp[o++] = idx[j++];
        }
        memcpy(idx, tmp, (size_t)m * sizeof(uint32_t));
        if (w > m / 2)
            break;
    }
}

int oracle_bwt(const uint8_t *x, uint64_t n, uint32_t block, uint8_t *L, uint32_t *primary)
{
    if (n == 0)
        return ORACLE_OK;
    if (block == 0)
        return ORACLE_ERR_INVALID_ARG;
    uint32_t *idx = (uint32_t *)malloc((size_t)block * sizeof(uint32_t));
    uint32_t *tmp = (uint32_t *)malloc((size_t)block * sizeof(uint32_t));
    if (!idx || !tmp) {
        free(idx);
        free(tmp);
        return ORACLE_ERR_CAPACITY;
    }
    uint64_t blocks = (n + block - 1) / block;
    for (uint64_t c = 0; c < blocks; ++c) {
        const uint8_t *b = x + c * block;
        uint32_t m = (uint32_t)(n - c * block < block ? n - c * block : block);
        for (uint32_t j = 0; j < m; ++j)
            idx[j] = j;
        sort_rotations(b, m, idx, tmp);
        for (uint32_t r = 0; r < m; ++r) {
            uint32_t j = idx[r];
            L[c * block + r] = b[j == 0 ? m - 1 : j - 1];
            if (j == 0)
                primary[c] = r;
        }
    }
    free(idx);
    free(tmp);
    return ORACLE_OK;
}

int oracle_ibwt(const uint8_t *L, uint64_t n, uint32_t block, const uint32_t *primary,
                uint8_t *out)
{
    if (n == 0)
        return ORACLE_OK;
    if (block == 0)
        return ORACLE_ERR_INVALID_ARG;
    uint32_t *lf = (uint32_t *)malloc((size_t)block * sizeof(uint32_t));
    if (!lf)
        return ORACLE_ERR_CAPACITY;
    uint64_t blocks = (n + block - 1) / block;
    for (uint64_t c = 0; c < blocks; ++c) {
        const uint8_t *l = L + c * block;
        uint32_t m = (uint32_t)(n - c * block < block ? n - c * block : block);
        if (primary[c] >= m) {
            free(lf);
            return ORACLE_ERR_CORRUPT;
        }
        /* first[v]: the first row of the sorted first column holding v */
        uint64_t cnt[256] = {0}, first[256];
        for (uint32_t p = 0; p < m; ++p)
            ++cnt[l[p]];
        uint64_t acc = 0;
        for (int v = 0; v < 256; ++v) {
            first[v] = acc;
            acc += cnt[v];
        }
        /* the k-th occurrence of v in the last column is the k-th in the
         * first column: row p's rotation, moved one byte back, is row lf[p] */
        uint64_t seen[256] = {0};
        for (uint32_t p = 0; p < m; ++p)
            lf[p] = (uint32_t)(first[l[p]] + seen[l[p]]++);
        uint32_t p = primary[c];
        for (uint32_t t = 0; t < m; ++t) {
            out[c * block + (m - 1 - t)] = l[p];
            p = lf[p];
        }
    }
    free(lf);
    return ORACLE_OK;
}

/* Move-to-front coding of each block (the stage that usually follows the
 * block-sorting transform: Burrows and Wheeler, 1994, Section 4): a list of
 * the 256 byte values, in increasing order at the start of every block; each
 * byte is coded as its current position in the list and then moved to the
 * front.  Runs of equal bytes become runs of zeros. */
int oracle_mtf(const uint8_t *x, uint64_t n, uint32_t block, uint8_t *out)
{
    if (n == 0)
        return ORACLE_OK;
    if (block == 0)
        return ORACLE_ERR_INVALID_ARG;
    uint8_t list[256];
    for (uint64_t i = 0; i < n; ++i) {
        if (i % block == 0)
            for (int v = 0; v < 256; ++v)
                list[v] = (uint8_t)v;
        const uint8_t c = x[i];
        int j = 0;
        while (list[j] != c)
            ++j;
        out[i] = (uint8_t)j;
        for (; j > 0; --j)
            list[j] = list[j - 1];
        list[0] = c;
    }
    return ORACLE_OK;
}

int oracle_imtf(const uint8_t *idx, uint64_t n, uint32_t block, uint8_t *out)
{
    if (n == 0)
        return ORACLE_OK;
    if (block == 0)
        return ORACLE_ERR_INVALID_ARG;
    uint8_t list[256];
    for (uint64_t i = 0; i < n; ++i) {
        if (i % block == 0)
            for (int v = 0; v < 256; ++v)
                list[v] = (uint8_t)v;
        int j = idx[i];
        const uint8_t c = list[j];
        out[i] = c;
        for (; j > 0; --j)
            list[j] = list[j - 1];
        list[0] = c;
    }
    return ORACLE_OK;
}
