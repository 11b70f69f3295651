// Codebook: the tree step of the paper's Huffman Method 1 (Section III-A) --
// the two lightest nodes are replaced by one internal node whose weight is
// their sum, until a single root remains; a leaf's depth is its code length.
// Then canonical codes in (length, byte value) order.
//
// One CTA of 256 threads, no host round trip:
//  1. rank sort of the present bytes by (weight, byte)            (parallel)
//  2. two-queue merge: sorted leaves in one queue, merged nodes appended to a
//     second one.  Merged weights never decrease and merged ids grow in
//     creation order, so the second queue is sorted by (weight, id) too; a
//     leaf wins a weight tie because every byte id < 256 <= any merged id.
//     This pops exactly the sequence of a (weight, id) min-heap.  (thread 0)
//  3. depths by pointer jumping over the parent links          (parallel)
//  4. the 32-bit limit check, then canonical codes with the RFC 1951
//     next_code recurrence and a per-length rank by byte value  (parallel)
#include "codebook_impl.cuh"

namespace huff {
namespace {

constexpr int kCbBlock = 256;

__global__ void __launch_bounds__(kCbBlock)
    k_build_codebook(const unsigned long long *__restrict__ hist, huff_codebook_t *__restrict__ cb,
                     int32_t *status, int limit, int limited)
{
    __shared__ cbk::CodebookShared sh;
    cbk::build_codebook(hist, cb, status, sh, limit, limited != 0);
}

}  // namespace

cudaError_t launch_build_codebook(const unsigned long long *d_hist, huff_codebook_t *d_cb,
                                  int32_t *d_status, cudaStream_t s, uint32_t limit)
{
    const bool limited = limit != 0;
    k_build_codebook<<<1, kCbBlock, 0, s>>>(d_hist, d_cb, d_status,
                                            limited ? (int)limit : (int)kMaxCodeLen, limited);
    return cudaGetLastError();
}

}  // namespace huff
