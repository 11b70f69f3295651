// Batched engine internals shared by batch.cu (kernels, plans) and
// server.cu (served rounds).
#pragma once

#include <vector>

#include "huff_internal.cuh"

namespace huff {

constexpr int kBatchBlock = 256;
constexpr int kBatchWarps = kBatchBlock / 32;
// The encode and decode phases run each half of a CTA on its own items
// (its own code or lookup table), so that small buffers leave fewer warps
// idle than with items of the whole CTA.
constexpr int kHalf = kBatchBlock / 2;
constexpr int kHalfWarps = kBatchWarps / 2;
constexpr int kUnitsPerItem = kHalfWarps;  // encode: one unit per warp of a half
constexpr int kTasksPerItem = kHalfWarps;  // decode: one task per warp of a half

// control words (device): barrier arrivals and generation, then tickets
enum { kCtlArrive = 0, kCtlGen = 1, kCtlTicket0 = 2, kCtlWords = 8 };

struct BatchBuf {
    const uint8_t *in;
    uint64_t in_bytes;
    uint8_t *out;
    uint64_t out_cap;
    unsigned long long *out_bytes;
    int32_t *status;
};

struct BatchArgs {
    const BatchBuf *bufs;
    uint32_t count;
    uint32_t cs;                    // compress: chunk symbols
    const uint64_t *unit_base;      // compress: [count + 1] prefix of units
    const uint64_t *item_base;      // compress: [count + 1] prefix of encode items
    uint16_t *unit_hist;            // compress: [units][256]
    unsigned long long *unit_off;   // compress: per buffer units_b + 1 entries at unit_base[b] + b
    huff_codebook_t *cbs;           // compress: [count]
    uint4 *unit_owner;              // compress: [units] (its first input byte, low and high
                                    //   words; its bytes; its buffer), set in phase 0
    uint4 *item_owner;              // compress: [items] (buffer, item within it, its first
                                    //   unit's index in unit_base order, low and high words)
    uint64_t *dec_items;            // decompress: [count + 1] items, then their prefix
    uint32_t min_lanes;             // decompress: lanes per buffer to aim for
    unsigned int *ctl;              // kCtlWords
    int32_t *fail;                  // whole-batch failure (barrier timeout)
    uint32_t barrier_extra;         // test hook: CTAs the barriers wait for beyond the grid
};

// Host-side description of a batch's device block (see batch_layout).
struct BatchLayout {
    uint32_t count;
    huff_op_t op;
    std::vector<BatchBuf> bufs;
    std::vector<uint64_t> unit_base, item_base;
    uint64_t o_ctl, o_bufs, o_ub, o_ib, o_di, o_uh, o_uo, o_cb, o_uw, o_iw;
    uint64_t bytes;         // device block size
    uint64_t upload_bytes;  // leading part filled from the host
};

void batch_layout(const huff_batch_desc_t *descs, uint32_t count, huff_op_t op, BatchLayout &L);
BatchArgs batch_args(const BatchLayout &L, void *d_block, uint32_t cs, uint32_t lanes,
                     uint32_t barrier_extra = 0);
cudaError_t batch_upload(const BatchLayout &L, void *d_block, uint8_t *host, cudaStream_t s);
int batch_occupancy(huff_op_t op);
cudaError_t batch_launch(huff_op_t op, const BatchArgs &args, unsigned grid, cudaStream_t s);
huff_status_t batch_check(const huff_batch_desc_t *descs, uint32_t count, huff_op_t op,
                          const huff_batch_params_t &prm);

}  // namespace huff
