/*
 * huff.h -- C ABI of the GB300 Huffman library (libhuff.so).
 *
 * The library runs the data-parallel hot path of the Huffman scheme of
 * "Parallel Data Compression Techniques" (Noel, Graham, Liu), Section III-A:
 *
 *   Method 1: count how often each byte occurs, build the weighted binary
 *   tree by repeatedly replacing the two lightest nodes with one internal
 *   node whose weight is their sum, and code each byte by its leaf's path.
 *   Method 2: cut the data into segments with ids, code them independently
 *   and reassemble them by id.
 *
 * Here the segments are fixed chunks of `chunk_symbols` bytes whose starting
 * bit offsets are stored in the stream, so every chunk decodes on its own.
 *
 * Conventions shared by every call:
 *  - Pointers named d_* are DEVICE pointers, owned by the caller.  The plain
 *    calls never allocate; scratch comes from the caller (d_ws).
 *  - d_in, d_out and d_stream must be 16-byte aligned (cudaMalloc and torch
 *    allocations are); otherwise HUFF_ERR_INVALID_ARG is returned.
 *  - Calls are asynchronous on `stream` (0 = the legacy default stream).
 *    The RETURN VALUE reports argument and launch errors only.
 *  - Errors found on the device (code too long, corrupt stream, capacity,
 *    wait timeout) are written to *d_status with "first error wins".  The
 *    caller sets *d_status = 0 before the first call of a chain (for example
 *    build_codebook -> encode); every kernel reads it first and does nothing
 *    if it is already non-zero, so a failed step stops the rest of the chain.
 *    huff_compress clears *d_status itself.  Read it after synchronising.
 *
 * Stream layout (all integers little-endian):
 *   [0, 256)            code length of each byte value, u8 (0 = absent)
 *   [256, 264)          n, the number of symbols, u64
 *   [264, 268)          chunk_symbols, u32
 *   [268, 272)          longest code length, u32
 *   [272, 272 + 8C)     bit offset of each chunk in the payload, u64,
 *                       C = ceil(n / chunk_symbols)
 *   then                payload as u32 words; payload bit j is bit
 *                       (31 - j % 32) of word j / 32 (most significant bit
 *                       first), the last word zero padded.
 *
 * Codes: lengths from the merge tree with ties broken by (weight, id), leaf
 * id = byte value and merged nodes numbered 256, 257, ... in creation order;
 * canonical codes in (length, byte value) order.  One distinct byte gets the
 * 1-bit code "0".  A code longer than 32 bits is an error, not limited.
 */
#ifndef HUFF_H
#define HUFF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t huff_status_t;

#define HUFF_OK 0
#define HUFF_ERR_INVALID_ARG (-1)    /* bad argument (host) / symbol or size (device) */
#define HUFF_ERR_CODE_TOO_LONG (-2)  /* a code would need more than 32 bits           */
#define HUFF_ERR_CAPACITY (-3)       /* output buffer too small                       */
#define HUFF_ERR_CORRUPT_STREAM (-4) /* stream fails validation                       */
#define HUFF_ERR_CUDA (-5)           /* a CUDA call or launch failed                  */
#define HUFF_ERR_TIMEOUT (-6)        /* a bounded device wait gave up                 */
#define HUFF_ERR_BUDGET (-7)         /* request can never fit the memory budget       */
#define HUFF_ERR_UNSUPPORTED (-8)    /* no usable device / unsupported configuration  */

#define HUFF_HEADER_BYTES 272u
#define HUFF_DEFAULT_CHUNK_SYMBOLS 16384u
#define HUFF_MIN_CHUNK_SYMBOLS 16u
#define HUFF_MAX_CHUNK_SYMBOLS (1u << 24)
#define HUFF_MAX_CODE_LEN 32u

/* The CUDA stream type, declared without including cuda_runtime.h. */
typedef struct CUstream_st *huff_stream_t;

/* Codebook, plain data, 1288 bytes; lives in device memory for the calls. */
typedef struct huff_codebook {
    uint8_t len[256];   /* code length of each byte value, 0 = absent      */
    uint32_t code[256]; /* canonical code, right-aligned in the low bits   */
    uint32_t nsym;      /* number of byte values with a code               */
    uint32_t max_len;   /* longest code length                             */
} huff_codebook_t;

/* Text of a status code; never NULL. */
const char *huff_status_str(huff_status_t status);

/* Library version, major * 10000 + minor * 100 + patch. */
int huff_version(void);

/* Upper bound on the stream size of n input bytes coded with a codebook from
 * huff_build_codebook: header + 8 * ceil(n / chunk_symbols) + 4 * ceil(n / 4)
 * + 4.  It holds because an optimal code never spends more than 8 bits per
 * byte on average (and 1 bit per byte with one distinct byte), so no read
 * back is needed to size the output.  Returns 0 for an invalid
 * chunk_symbols. */
uint64_t huff_max_stream_size(uint64_t n, uint32_t chunk_symbols);

/* Bytes of scratch (d_ws) that huff_encode and huff_compress need for n
 * bytes.  Returns 0 for an invalid chunk_symbols. */
uint64_t huff_workspace_size(uint64_t n, uint32_t chunk_symbols);

/* Method 1, first step (Section III-A): d_hist[b] = number of bytes equal to
 * b in d_in[0, n).  d_hist is u64[256]; the call clears it first.
 * Errors: HUFF_ERR_INVALID_ARG (null or misaligned pointers),
 * HUFF_ERR_CUDA. */
huff_status_t huff_histogram(const uint8_t *d_in, uint64_t n, uint64_t *d_hist,
                             huff_stream_t stream);

/* Bytes of per-unit histograms that huff_histogram_units writes for n input
 * bytes: 512 (u16[256]) per 16384-byte unit. */
uint64_t huff_unit_hist_size(uint64_t n);

/* huff_histogram plus every 16384-byte unit's own histogram, u16[256] per
 * unit, into d_unit_hist (huff_unit_hist_size(n) bytes, 16-byte aligned).
 * huff_encode_units turns them into each unit's bit offset (a dot product
 * with the code lengths), which spares the encoder a counting pass over the
 * input.  Errors as huff_histogram. */
huff_status_t huff_histogram_units(const uint8_t *d_in, uint64_t n, uint64_t *d_hist,
                                   uint16_t *d_unit_hist, huff_stream_t stream);

/* Method 1, tree step (Section III-A): from d_hist (u64[256]) build the code
 * lengths with the (weight, id) merge tree, then the canonical codes, into
 * *d_cb.  One CTA; no host synchronisation.  Device errors in *d_status:
 * HUFF_ERR_CODE_TOO_LONG (then *d_cb is all zero).  Returns
 * HUFF_ERR_INVALID_ARG for null pointers, HUFF_ERR_CUDA on launch failure. */
huff_status_t huff_build_codebook(const uint64_t *d_hist, huff_codebook_t *d_cb,
                                  int32_t *d_status, huff_stream_t stream);

/* Length-limited codebook (an extension of the tree step, not in the
 * paper): the code lengths are the Huffman lengths of huff_build_codebook
 * when none exceeds max_len, else the optimal lengths of at most max_len
 * bits by package-merge (Larmore & Hirschberg 1990; the present bytes sorted
 * by (weight, byte), a byte before a package of equal weight).  Canonical
 * codes as above.  max_len in 1..32 (else HUFF_ERR_INVALID_ARG); more
 * distinct bytes than 2^max_len is HUFF_ERR_CODE_TOO_LONG in *d_status.
 * With max_len <= 12 every code fits the decoder's lookup table. */
huff_status_t huff_build_codebook_limited(const uint64_t *d_hist, uint32_t max_len,
                                          huff_codebook_t *d_cb, int32_t *d_status,
                                          huff_stream_t stream);

/* Encode d_in[0, n) with *d_cb into the stream layout above at d_out.
 * Method 1's coding step with Method 2's segments as chunks of
 * chunk_symbols bytes (a multiple of 16 in [16, 2^24]).
 *  - *d_out_bytes receives the exact stream size (also on a capacity
 *    error, so the caller can retry with a larger buffer).
 *  - out_cap: bytes available at d_out; huff_max_stream_size(n,
 *    chunk_symbols) always suffices for a codebook built from d_in.
 *  - d_ws / ws_bytes: scratch of at least huff_workspace_size(n,
 *    chunk_symbols) bytes, 16-byte aligned; its contents are clobbered.
 *  - Precondition: every byte value present in d_in has a code in *d_cb
 *    (always true for a codebook built from d_in's histogram); otherwise
 *    the stream is unspecified.
 * Device errors: HUFF_ERR_CAPACITY, HUFF_ERR_TIMEOUT.  Host errors:
 * HUFF_ERR_INVALID_ARG, HUFF_ERR_CUDA.  Calls sharing one d_ws must not
 * overlap on the GPU. */
huff_status_t huff_encode(const uint8_t *d_in, uint64_t n, const huff_codebook_t *d_cb,
                          uint32_t chunk_symbols, uint8_t *d_out, uint64_t out_cap,
                          uint64_t *d_out_bytes, void *d_ws, uint64_t ws_bytes,
                          int32_t *d_status, huff_stream_t stream);

/* huff_encode for a codebook built from the same input, with the unit
 * histograms of huff_histogram_units(d_in, n, ...): same arguments, result
 * and errors, one input read fewer. */
huff_status_t huff_encode_units(const uint8_t *d_in, uint64_t n, const huff_codebook_t *d_cb,
                                const uint16_t *d_unit_hist, uint32_t chunk_symbols,
                                uint8_t *d_out, uint64_t out_cap, uint64_t *d_out_bytes,
                                void *d_ws, uint64_t ws_bytes, int32_t *d_status,
                                huff_stream_t stream);

/* Largest input huff_encode_noalloc accepts (1 GiB). */
#define HUFF_NOALLOC_MAX_SYMBOLS (1ull << 30)

/* huff_encode for callers that cannot allocate device memory while they
 * encode -- for example a latency-critical loop where an allocation would
 * synchronise the device, a service that runs inside a fixed memory budget
 * reserved at start-up, or a wrapper that only ever hands over input and
 * output buffers.  It takes no workspace: the encoder's scratch (bit count
 * and bit offset of each 16 KiB unit) is a fixed array inside the library,
 * about 0.75 MiB of device memory that every GPU which loads the library
 * keeps until the process exits.  The paper has no counterpart; this is a
 * deployment variant of huff_encode with the same arguments minus
 * d_ws / ws_bytes, the same stream and the same device errors.
 *  - n above HUFF_NOALLOC_MAX_SYMBOLS -> HUFF_ERR_BUDGET, nothing launched.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.
 *  - All calls share the one array: each call rewrites the entries it reads,
 *    but calls that overlap on the GPU (other streams, other threads) race
 *    on it and must be serialised by the caller.
 * Host errors: HUFF_ERR_INVALID_ARG, HUFF_ERR_CUDA, HUFF_ERR_UNSUPPORTED. */
huff_status_t huff_encode_noalloc(const uint8_t *d_in, uint64_t n, const huff_codebook_t *d_cb,
                                  uint32_t chunk_symbols, uint8_t *d_out, uint64_t out_cap,
                                  uint64_t *d_out_bytes, int32_t *d_status,
                                  huff_stream_t stream);

/* Decode the stream d_stream[0, stream_bytes) into d_out[0, n) (Method 2's
 * reassembly by chunk id; the code is lossless).  The stream is validated:
 * header fields, a complete code (sum of 2^-len == 1, or one code of length
 * 1), off[0] == 0, non-decreasing offsets within the payload, no chunk
 * reading past the next chunk's offset and every chunk but the last ending
 * exactly on it.  Any failure -> HUFF_ERR_CORRUPT_STREAM in *d_status; n
 * larger than out_cap -> HUFF_ERR_CAPACITY.  *d_n receives n once the header
 * is valid.  Trailing bytes after the payload are ignored.
 * Host errors: HUFF_ERR_INVALID_ARG, HUFF_ERR_CUDA. */
huff_status_t huff_decode(const uint8_t *d_stream, uint64_t stream_bytes, uint8_t *d_out,
                          uint64_t out_cap, uint64_t *d_n, int32_t *d_status,
                          huff_stream_t stream);

/* Method 1 end to end on one stream, no host synchronisation: clear
 * *d_status, huff_histogram_units, huff_build_codebook and
 * huff_encode_units, with the histograms and codebook kept in d_ws
 * (ws_bytes >= huff_workspace_size).  Same arguments and errors as
 * huff_encode. */
huff_status_t huff_compress(const uint8_t *d_in, uint64_t n, uint32_t chunk_symbols,
                            uint8_t *d_out, uint64_t out_cap, uint64_t *d_out_bytes,
                            void *d_ws, uint64_t ws_bytes, int32_t *d_status,
                            huff_stream_t stream);

/* ---------------------------------------------------------------------
 * Batched engine.  The paper's Method 2 (Section III-A) compresses every
 * segment independently with its own tree and reassembles the results by
 * segment id; here each descriptor is one independent buffer with its own
 * codebook and stream, and a whole batch runs as one persistent fused
 * launch (histograms, codebooks and unit offsets, encode -- or header
 * scan and decode) captured once in a CUDA graph.  Every buffer's stream is
 * byte-identical to huff_compress on that buffer alone.
 * ------------------------------------------------------------------- */
typedef enum huff_op { HUFF_BATCH_COMPRESS = 0, HUFF_BATCH_DECOMPRESS = 1 } huff_op_t;

typedef struct huff_batch_desc {
    const uint8_t *d_in;   /* compress: input bytes; decompress: one stream  */
    uint64_t in_bytes;     /* compress: n; decompress: stream bytes          */
    uint8_t *d_out;        /* compress: stream; decompress: decoded bytes    */
    uint64_t out_cap;      /* bytes available at d_out                       */
    uint64_t *d_out_bytes; /* compress: stream size; decompress: n           */
    int32_t *d_status;     /* this buffer's device status, cleared each run  */
} huff_batch_desc_t;

typedef struct huff_batch_params {
    uint32_t chunk_symbols; /* compress: chunk size of every stream           */
    uint32_t ctas_per_sm;   /* persistent CTAs per SM, 0 = as many as fit     */
    uint32_t decode_lanes;  /* decompress: lanes to spread a buffer over
                               (1..65536): its chunks are split into the
                               smallest power of two S <= 32 of sub-segments
                               with chunks x S >= decode_lanes            */
    uint32_t use_graph;     /* capture the launch in a CUDA graph (1) or not  */
    uint32_t barrier_extra; /* test hook, 0 in use: nonzero makes the launch's
                               grid barriers wait for that many CTAs more than
                               exist, so every wait runs out and the buffers
                               report HUFF_ERR_TIMEOUT (exercises the bounded
                               waits without a GPU fault)                    */
} huff_batch_params_t;

typedef struct huff_batch_plan huff_batch_plan_t; /* opaque */

/* Defaults: 16384-symbol chunks, full occupancy, 128 decode lanes, graph on. */
void huff_batch_default_params(huff_batch_params_t *params);

/* Plan a batch of `count` buffers for `op` (params may be NULL for the
 * defaults).  The plan copies the descriptors, allocates its own device
 * metadata and scratch (per-unit histograms, codebooks, offsets: about
 * 520 bytes per 16 KiB of input for compression) and captures the launch in
 * a CUDA graph; runs then allocate nothing.  Buffers are 16-byte aligned;
 * compress outputs need out_cap >= header + offset table (use
 * huff_max_stream_size).  Errors: HUFF_ERR_INVALID_ARG, HUFF_ERR_CUDA. */
huff_status_t huff_batch_plan(const huff_batch_desc_t *descs, uint32_t count, huff_op_t op,
                              const huff_batch_params_t *params, huff_batch_plan_t **plan);

/* Run the planned batch on `stream`, asynchronously.  Per-buffer results
 * and errors land in each descriptor's d_out_bytes and d_status (a wait
 * that gave up marks every buffer HUFF_ERR_TIMEOUT).  Runs of one plan must
 * not overlap on the GPU. */
huff_status_t huff_batch_run(huff_batch_plan_t *plan, huff_stream_t stream);

/* The parameters a plan uses, its grid size and whether it runs as a graph. */
huff_status_t huff_batch_info(const huff_batch_plan_t *plan, huff_batch_params_t *params,
                              uint32_t *grid, int32_t *used_graph);

/* ---- segmented container: one codebook per segment ----------------------
 * The paper's Method 2 taken literally (Section III-A): the input is cut into
 * segments with ids, each segment is coded with its own tree, and the
 * decoder reassembles them by id.  Container layout (all integers LE):
 *   [0, 8)   n, the total number of bytes
 *   [8, 16)  segment_bytes (a multiple of 16; the last segment may be shorter)
 *   [16, 24) count = ceil(n / segment_bytes)
 *   [24, 24 + 8 (count + 1))  start[i]: byte offset of segment i's stream;
 *            start[count] is the container size
 *   then the streams: segment i's stream (the layout above, its own lengths
 *   and offsets) at start[i], a multiple of 16; start[0] = the header size
 *   rounded up to 16; zero bytes between streams.
 * Both calls run the batched engine (one fused launch) and SYNCHRONIZE the
 * stream: they plan the batch on the host and free the plan afterwards.
 * Both ALLOCATE device memory on every call (cudaMalloc / cudaFree: the
 * batch plan's descriptor block, and for decompression 12 bytes of scratch
 * per segment); callers that must not allocate while they run keep a
 * persistent plan over the segments with huff_batch_plan / huff_batch_run.
 * Decompression spreads each segment over enough lanes that the whole
 * container fills about one wave of decoders (256 lanes per SM). */
uint64_t huff_segmented_max_size(uint64_t n, uint64_t segment_bytes, uint32_t chunk_symbols);
/* Device scratch of huff_segmented_compress: the streams in worst-case
 * slots, then per-segment sizes and statuses. */
uint64_t huff_segmented_workspace_size(uint64_t n, uint64_t segment_bytes,
                                       uint32_t chunk_symbols);
/* Compress d_in[0, n) into the container at d_out.  *d_status is cleared
 * first; *d_out_bytes receives the container size; device errors (the first
 * of any segment, or HUFF_ERR_CAPACITY when the container exceeds out_cap)
 * in *d_status.  out_cap must hold at least the header and start table.
 * d_in, d_out, d_ws 16-byte aligned.  Host errors: HUFF_ERR_INVALID_ARG,
 * HUFF_ERR_CUDA. */
huff_status_t huff_segmented_compress(const uint8_t *d_in, uint64_t n, uint64_t segment_bytes,
                                      uint32_t chunk_symbols, uint8_t *d_out, uint64_t out_cap,
                                      uint64_t *d_out_bytes, void *d_ws, uint64_t ws_bytes,
                                      int32_t *d_status, huff_stream_t stream);
/* Decompress a container (read on the host first: header and start table)
 * into d_out[0, n).  *d_n receives n once the header is valid.  A malformed
 * header or table, or a segment that fails or decodes to a size other than
 * its own, is HUFF_ERR_CORRUPT_STREAM in *d_status; n > out_cap is
 * HUFF_ERR_CAPACITY.  d_in 16-byte aligned.  Host errors:
 * HUFF_ERR_INVALID_ARG, HUFF_ERR_CUDA. */
huff_status_t huff_segmented_decompress(const uint8_t *d_in, uint64_t in_bytes, uint8_t *d_out,
                                        uint64_t out_cap, uint64_t *d_n, int32_t *d_status,
                                        huff_stream_t stream);

/* ---- Method 3: block-sorting transform, then Method 2 ------------------
 * Method 3 (Section III-A) runs the Burrows-Wheeler transform over each
 * block of the data and then Method 2's coder over the result.  Reading of
 * the transform (the paper's one-line description is garbled): blocks are
 * runs of `block` consecutive bytes (the last may be shorter), transformed
 * independently; a block's m cyclic rotations are sorted by unsigned byte
 * value, equal rotations (periodic blocks) in the order of their starts;
 * the output is the last byte of every rotation in sorted order and the
 * primary index, the sorted row of the rotation starting at the block's
 * first byte (Burrows and Wheeler, 1994).
 * Limits: 1 <= block, n <= HUFF_BWT_MAX_N.  Both calls SYNCHRONIZE the
 * stream (the forward transform reads a count back after every doubling
 * round).  Device buffers: d_in / d_last n bytes, d_primary one u32 per
 * block (ceil(n / block)); the workspace is huff_bwt_workspace_size bytes,
 * 16-byte aligned, owned by the caller (about 60 n bytes).
 * Errors: host HUFF_ERR_INVALID_ARG / HUFF_ERR_CUDA; the inverse puts
 * HUFF_ERR_CORRUPT_STREAM in *d_status when a primary index lies outside
 * its block (the output is then not written). */
#define HUFF_BWT_MAX_N 2147483647ull
uint64_t huff_bwt_workspace_size(uint64_t n, uint32_t block);
huff_status_t huff_bwt_forward(const uint8_t *d_in, uint64_t n, uint32_t block, uint8_t *d_last,
                               uint32_t *d_primary, void *d_ws, uint64_t ws_bytes,
                               int32_t *d_status, huff_stream_t stream);
huff_status_t huff_bwt_inverse(const uint8_t *d_last, uint64_t n, uint32_t block,
                               const uint32_t *d_primary, uint8_t *d_out, void *d_ws,
                               uint64_t ws_bytes, int32_t *d_status, huff_stream_t stream);
/* Move-to-front coding per block (Method 3's optional second stage; Burrows
 * and Wheeler 1994, Section 4): every block of `block` bytes starts from the
 * list 0..255; each byte is coded as its position in the list and moved to
 * the front; the inverse decodes.  Asynchronous on the stream; d_in / d_out
 * n bytes (they may be the same buffer); workspace huff_mtf_workspace_size
 * bytes, 16-byte aligned: 516 bytes per 1 KiB segment of every block (the
 * segments' distinct bytes, counts and starting lists) plus n, so about
 * 1.5 n.  Host errors only:
 * HUFF_ERR_INVALID_ARG, HUFF_ERR_CUDA. */
uint64_t huff_mtf_workspace_size(uint64_t n, uint32_t block);
huff_status_t huff_mtf_forward(const uint8_t *d_in, uint64_t n, uint32_t block, uint8_t *d_out,
                               void *d_ws, uint64_t ws_bytes, huff_stream_t stream);
huff_status_t huff_mtf_inverse(const uint8_t *d_in, uint64_t n, uint32_t block, uint8_t *d_out,
                               void *d_ws, uint64_t ws_bytes, huff_stream_t stream);
/* Method 3 container (all integers LE):
 *   [0, 8) n; [8, 12) block; [12, 16) count = ceil(n / block);
 *   [16, 20) stages: bit 0 set = move-to-front after the transform (other
 *   bits zero); [20, 20 + 4 count) primary index of every block; zero bytes
 *   up to a multiple of 16; then the segmented container (above) of the
 *   transformed (and move-to-front coded) bytes, with its own segment size
 *   and chunk size.
 * huff_m3_compress: *d_out_bytes receives the container size; workspace
 * huff_m3_workspace_size (16-byte aligned, d_out too).  huff_m3_decompress
 * reads the header on the host, decodes the segments into the workspace
 * (huff_m3_decompress_workspace_size(n, block) bytes, n and block from the
 * header) and inverts the transform into d_out; a malformed header, a
 * segment error or a segmented container that does not hold n bytes is
 * HUFF_ERR_CORRUPT_STREAM in *d_status, n > out_cap HUFF_ERR_CAPACITY.
 * Both SYNCHRONIZE the stream. */
uint64_t huff_m3_max_size(uint64_t n, uint32_t block, uint64_t segment_bytes,
                          uint32_t chunk_symbols);
uint64_t huff_m3_workspace_size(uint64_t n, uint32_t block, uint64_t segment_bytes,
                                uint32_t chunk_symbols);
#define HUFF_M3_MTF 1u /* stages: move-to-front after the transform */
huff_status_t huff_m3_compress(const uint8_t *d_in, uint64_t n, uint32_t block,
                               uint64_t segment_bytes, uint32_t chunk_symbols, uint32_t stages,
                               uint8_t *d_out, uint64_t out_cap, uint64_t *d_out_bytes,
                               void *d_ws, uint64_t ws_bytes, int32_t *d_status,
                               huff_stream_t stream);
uint64_t huff_m3_decompress_workspace_size(uint64_t n, uint32_t block);
huff_status_t huff_m3_decompress(const uint8_t *d_in, uint64_t in_bytes, uint8_t *d_out,
                                 uint64_t out_cap, uint64_t *d_n, void *d_ws, uint64_t ws_bytes,
                                 int32_t *d_status, huff_stream_t stream);

/* Autotuner.  Times candidate parameter sets on the caller's own batch and
 * returns the fastest in *best; results are cached per device, operation
 * and batch shape (buffer count, total and mean size in powers of two, and
 * for decompression nothing else), so a later call for a batch of the same
 * shape returns at once.  Candidates:
 *   decompress: decode_lanes in {32, 64, 128, 256} x ctas_per_sm in
 *               {as many as fit, 1};
 *   compress:   chunk_symbols in {base, 4096} (the chunk size of every
 *               stream; 4096 only if every out_cap holds
 *               huff_max_stream_size(n, 4096)) x ctas_per_sm in {as many as
 *               fit, 1}, with flags & HUFF_TUNE_ROUND_TRIP scored by the
 *               compress time plus the best decompress time of the streams
 *               it produced (decode_lanes tuned alongside), else by the
 *               compress time alone.
 * `base` (NULL = defaults) supplies everything not tuned.  Tuning RUNS the
 * batch several times on `stream` (the outputs are overwritten with valid
 * results each time) and synchronizes it; with HUFF_TUNE_ROUND_TRIP it also
 * allocates, and frees again, scratch for the decoded bytes.  With the
 * environment variable HUFF_TUNE_CACHE naming a file, the cache persists
 * there as JSON lines (device name/SM count, op, shape buckets, chunk size,
 * round trip, and the chosen chunk_symbols, ctas_per_sm, decode_lanes): the
 * file is read on the first call and a line is appended per newly tuned
 * shape; lines that do not parse or hold values the tuner cannot choose are
 * ignored.  Errors: those of huff_batch_plan / huff_batch_run,
 * HUFF_ERR_CUDA. */
#define HUFF_TUNE_FORCE 1u      /* ignore the cache and tune again */
#define HUFF_TUNE_ROUND_TRIP 2u /* compress: score by compress + decompress */
huff_status_t huff_batch_autotune(const huff_batch_desc_t *descs, uint32_t count, huff_op_t op,
                                  const huff_batch_params_t *base, uint32_t flags,
                                  huff_batch_params_t *best, huff_stream_t stream);

/* Free a plan (NULL is ignored).  Its runs must have completed. */
void huff_batch_destroy(huff_batch_plan_t *plan);

/* ---------------------------------------------------------------------
 * Served path: compress and decompress requests of mixed sizes arrive at
 * any time; a scheduler thread admits them into rounds (continuous
 * batching) as round slots and device memory free up, each round being one
 * fused batch launch on its own stream, so admitted work overlaps on the
 * device.  Device memory comes from one arena of `device_budget` bytes
 * reserved at creation; a request is admitted only when its input, output
 * and scratch fit.  Every result equals the same request served alone.
 * ------------------------------------------------------------------- */
typedef struct huff_server huff_server_t; /* opaque */

typedef struct huff_server_cfg {
    uint64_t device_budget;  /* arena bytes (default 8 GiB)                     */
    uint32_t max_rounds;     /* rounds in flight at once (default 3, max 16)    */
    uint32_t max_batch;      /* requests per round (default 256)                */
    uint32_t chunk_symbols;  /* chunk size of the streams written (16384)      */
    uint32_t decode_lanes;   /* lanes to spread a decompress request over, at
                                least (128; 1..65536): a round of few
                                requests spreads each over more, so that
                                the round fills about one wave of decoders */
} huff_server_cfg_t;

typedef struct huff_request {
    int32_t op;            /* HUFF_BATCH_COMPRESS or HUFF_BATCH_DECOMPRESS       */
    const uint8_t *h_in;   /* host input (pinned for full copy speed)           */
    uint64_t in_bytes;     /* input bytes (a whole stream for decompress)       */
    uint8_t *h_out;        /* host output                                        */
    uint64_t out_cap;      /* bytes available at h_out                           */
} huff_request_t;

typedef struct huff_result {
    int32_t done;       /* 1 once the result is in h_out                         */
    int32_t status;     /* HUFF_OK or the request's error                        */
    uint64_t out_bytes; /* stream size (compress) or n (decompress)             */
    double t_submit;    /* seconds since the server started: submitted,         */
    double t_start;     /*   admitted into a round,                              */
    double t_done;      /*   result copied out                                   */
} huff_result_t;

/* Defaults listed in huff_server_cfg_t. */
void huff_server_default_config(huff_server_cfg_t *cfg);

/* Start a server on the current device (cfg may be NULL).  Reserves the
 * arena and the pinned staging buffers, then starts the scheduler thread.
 * Errors: HUFF_ERR_INVALID_ARG, HUFF_ERR_CUDA. */
huff_status_t huff_server_create(const huff_server_cfg_t *cfg, huff_server_t **server);

/* Queue a request; *ticket identifies it.  Host buffers must stay valid
 * until the result is done.  HUFF_ERR_BUDGET when the request could never
 * fit the arena (it is not queued); HUFF_ERR_INVALID_ARG for bad fields. */
huff_status_t huff_server_submit(huff_server_t *server, const huff_request_t *req,
                                 uint64_t *ticket);

/* Non-blocking state of a request (res->done tells whether it finished). */
huff_status_t huff_server_poll(huff_server_t *server, uint64_t ticket, huff_result_t *res);

/* Wait up to timeout_ms for a request; HUFF_ERR_TIMEOUT if still running. */
huff_status_t huff_server_wait(huff_server_t *server, uint64_t ticket, uint32_t timeout_ms,
                               huff_result_t *res);

/* Forget a finished request (its ticket becomes invalid). */
huff_status_t huff_server_release(huff_server_t *server, uint64_t ticket);

/* Finish the queued and running requests, stop the thread, free everything. */
void huff_server_destroy(huff_server_t *server);

/* ---- LZSS Method 2: segmented LZSS (Section III-B) ------------------------
 * The data is cut into equal segments of segment_bytes (the last may be
 * shorter), each coded on its own against a sliding window of its most
 * recent bits; the segments' code lengths and codes are packed together.
 * The paper counts the window and match lengths in bits ("1024/24/12/8":
 * a 1024-bit window, matches of 12..24 bits, 8-bit literal blocks).
 * Readings: bits are read most significant bit of each byte first; the
 * window starts from the counting numbers (dict = 1: bytes 0, 1, 2, ...
 * before the segment) or from the segment's first `window` bits, stored as
 * they are (dict = 2; then no match reaches before the segment); at each
 * position the longest match of min_len .. min(max_len, bits left) bits is
 * taken, the smallest distance among equally long ones, and the source may
 * run into the bits being coded; a match is the bit 1, distance - 1 in
 * log2(window) bits and length - min_len in ceil(log2(max_len - min_len +
 * 1)) bits, a literal the bit 0 and the next min(block, bits left) bits.
 * Container (integers LE): [0,8) n; [8,16) segment_bytes; [16,20) window;
 * [20,24) min_len; [24,28) max_len; [28,32) block; [32,36) dict; [36,40)
 * zero; [40,48) count = ceil(n / segment_bytes); count u32 code lengths in
 * bits; then segment i's code, MSB first in bytes, from a 16-byte boundary
 * (the first after the table), zero padded to the next 16-byte boundary. */
typedef struct {
    uint32_t window;  /* bits, a power of two in [2, 65536] */
    uint32_t min_len; /* shortest match, bits, >= 1 */
    uint32_t max_len; /* longest match, bits, min_len .. 32 */
    uint32_t block;   /* bits per literal, 1 .. 32 */
    uint32_t dict;    /* 1: counting numbers; 2: the first `window` bits stored */
} huff_lzss_params_t;
/* Capacity that always holds the container, and compression's device
 * workspace; 0 for invalid parameters or segment sizes (segment_bytes a
 * multiple of 16 in [16, 2^24]). */
uint64_t huff_lzss_max_size(uint64_t n, uint64_t segment_bytes, const huff_lzss_params_t *params);
uint64_t huff_lzss_workspace_size(uint64_t n, uint64_t segment_bytes,
                                  const huff_lzss_params_t *params);
/* Compress d_in[0, n) into the container at d_out.  Asynchronous on the
 * stream, no host synchronisation and no allocation: one warp per segment
 * codes into a worst-case slot of d_ws, one CTA lays out the header and
 * table, a gather moves the codes into place.  *d_status is cleared first;
 * *d_out_bytes receives the container size; HUFF_ERR_CAPACITY in *d_status
 * when it exceeds out_cap.  d_in, d_out, d_ws 16-byte aligned (the caller's
 * buffers).  Host errors: HUFF_ERR_INVALID_ARG, HUFF_ERR_CUDA. */
huff_status_t huff_lzss_compress(const uint8_t *d_in, uint64_t n, uint64_t segment_bytes,
                                 const huff_lzss_params_t *params, uint8_t *d_out,
                                 uint64_t out_cap, uint64_t *d_out_bytes, void *d_ws,
                                 uint64_t ws_bytes, int32_t *d_status, huff_stream_t stream);
/* Workspace of decompression for a container of in_bytes bytes. */
uint64_t huff_lzss_decompress_workspace_size(uint64_t in_bytes);
/* Decompress a container into d_out[0, n); asynchronous, no allocation.
 * *d_n receives n once the header and table are consistent; an
 * inconsistent header or table, a distance or length out of range, or a
 * segment whose tokens do not end exactly at its recorded length is
 * HUFF_ERR_CORRUPT_STREAM in *d_status (the output is then unspecified);
 * n > out_cap is HUFF_ERR_CAPACITY.  One thread decodes each segment.
 * d_in, d_out, d_ws 16-byte aligned.  Host errors: HUFF_ERR_INVALID_ARG,
 * HUFF_ERR_CUDA. */
huff_status_t huff_lzss_decompress(const uint8_t *d_in, uint64_t in_bytes, uint8_t *d_out,
                                   uint64_t out_cap, uint64_t *d_n, void *d_ws, uint64_t ws_bytes,
                                   int32_t *d_status, huff_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* HUFF_H */
