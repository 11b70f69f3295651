/*
 * huff_oracle.h -- plain CPU oracle of the Huffman hot path.
 * TEST INFRASTRUCTURE ONLY: tests, the smoke check and the benchmark's CPU
 * baseline use it; the CUDA library neither includes nor links it.
 */
#ifndef HUFF_ORACLE_H
#define HUFF_ORACLE_H
#include <stdint.h>

#define ORACLE_OK 0
#define ORACLE_ERR_INVALID_ARG (-1)
#define ORACLE_ERR_CODE_TOO_LONG (-2)
#define ORACLE_ERR_CAPACITY (-3)
#define ORACLE_ERR_CORRUPT (-4)

#define ORACLE_HEADER_BYTES 272
#define ORACLE_MAX_CODE_LEN 32
#define ORACLE_MIN_CHUNK 16
#define ORACLE_MAX_CHUNK (1u << 24)

void oracle_histogram(const uint8_t *x, uint64_t n, uint64_t hist[256]);
int oracle_code_lengths(const uint64_t hist[256], uint8_t len[256]);
int oracle_code_lengths_limited(const uint64_t hist[256], uint32_t limit, uint8_t len[256]);
void oracle_canonical_codes(const uint8_t len[256], uint32_t code[256]);
uint64_t oracle_max_stream_size(uint64_t n, uint32_t cs);
int oracle_chunk_offsets(const uint8_t *x, uint64_t n, uint32_t cs, const uint8_t len[256],
                         uint64_t *off, uint64_t *total_bits);
int oracle_pack_bits(const uint8_t *x, uint64_t m, const uint8_t len[256], uint32_t *words,
                     uint64_t nwords, uint64_t *bits);
int oracle_encode(const uint8_t *x, uint64_t n, uint32_t cs, const uint8_t len[256],
                  uint8_t *out, uint64_t cap, uint64_t *out_bytes);
int oracle_compress(const uint8_t *x, uint64_t n, uint32_t cs, uint8_t *out, uint64_t cap,
                    uint64_t *out_bytes);
int oracle_decode(const uint8_t *s, uint64_t bytes, uint8_t *out, uint64_t cap,
                  uint64_t *n_out);
/* Method 3: block-sorting transform (Burrows-Wheeler) per block */
int oracle_bwt(const uint8_t *x, uint64_t n, uint32_t block, uint8_t *L, uint32_t *primary);
int oracle_ibwt(const uint8_t *L, uint64_t n, uint32_t block, const uint32_t *primary,
                uint8_t *out);
/* Method 3's optional second stage: move-to-front coding per block */
int oracle_mtf(const uint8_t *x, uint64_t n, uint32_t block, uint8_t *out);
int oracle_imtf(const uint8_t *idx, uint64_t n, uint32_t block, uint8_t *out);
/* LZSS Method 1 (one segment) and Method 2 (segmented container); the
 * paper's Section III-B, readings Z1-Z7 in lzss_oracle.c */
typedef struct {
    uint32_t window;  /* W: window bits, a power of two in [2, 65536] */
    uint32_t min_len; /* Lmin: shortest match, bits */
    uint32_t max_len; /* Lmax: longest match, bits (<= 32) */
    uint32_t block;   /* B: bits per literal (<= 32) */
    uint32_t dict;    /* 1: counting-numbers window; 2: first W bits stored */
} oracle_lzss_params;
int oracle_lzss_params_ok(const oracle_lzss_params *P);
uint64_t oracle_lzss_max_bits(uint64_t m, const oracle_lzss_params *P);
int oracle_lzss_encode(const uint8_t *x, uint64_t m, const oracle_lzss_params *P, uint8_t *out,
                       uint64_t cap_bytes, uint64_t *bits_out);
int oracle_lzss_decode(const uint8_t *code, uint64_t code_bits, const oracle_lzss_params *P,
                       uint8_t *y, uint64_t m);
uint64_t oracle_lzss_segmented_max_size(uint64_t n, uint64_t seg, const oracle_lzss_params *P);
int oracle_lzss_segmented_compress(const uint8_t *x, uint64_t n, uint64_t seg,
                                   const oracle_lzss_params *P, uint8_t *out, uint64_t cap,
                                   uint64_t *out_bytes);
int oracle_lzss_segmented_decompress(const uint8_t *c, uint64_t bytes, uint8_t *out, uint64_t cap,
                                     uint64_t *n_out);
#endif
