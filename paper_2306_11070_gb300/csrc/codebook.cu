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
#include "huff_internal.cuh"

namespace huff {
namespace {

constexpr int kCbBlock = 256;

__global__ void __launch_bounds__(kCbBlock)
    k_build_codebook(const unsigned long long *__restrict__ hist, huff_codebook_t *__restrict__ cb,
                     int32_t *status)
{
    __shared__ unsigned long long w[256];
    __shared__ unsigned long long nw[511];  // [0,m): leaves by (weight, byte); [m,2m-1): merged
    __shared__ int16_t par[511];
    __shared__ int16_t dep[511];
    __shared__ int16_t anc[511];
    __shared__ uint8_t leaf_sym[256];
    __shared__ uint8_t len_s[256];
    __shared__ uint32_t bl[kMaxCodeLen + 1];
    __shared__ uint32_t next_code[kMaxCodeLen + 1];
    __shared__ int s_max;

    if (chain_failed(status))
        return;
    const int t = threadIdx.x;
    const unsigned long long wt = hist[t];
    w[t] = wt;
    len_s[t] = 0;
    if (t <= (int)kMaxCodeLen)
        bl[t] = 0;
    if (t == 0)
        s_max = 0;
    const int present = wt > 0;
    const int m = __syncthreads_count(present);

    // 1. rank of byte t among present bytes, ordered by (weight, byte)
    if (present) {
        int rank = 0;
        for (int j = 0; j < 256; ++j) {
            const unsigned long long wj = w[j];
            rank += (wj > 0) & ((wj < wt) | ((wj == wt) & (j < t)));
        }
        leaf_sym[rank] = (uint8_t)t;
        nw[rank] = wt;
    }
    __syncthreads();

    if (m >= 2) {
        // 2. two-queue merge
        if (t == 0) {
            int li = 0, ii = m, ni = m;
            for (int step = 0; step < m - 1; ++step) {
                int a, b;
                if (li < m && (ii >= ni || nw[li] <= nw[ii]))
                    a = li++;
                else
                    a = ii++;
                if (li < m && (ii >= ni || nw[li] <= nw[ii]))
                    b = li++;
                else
                    b = ii++;
                nw[ni] = nw[a] + nw[b];
                par[a] = (int16_t)ni;
                par[b] = (int16_t)ni;
                ++ni;
            }
            par[2 * m - 2] = (int16_t)(2 * m - 2);  // the root points at itself
        }
        __syncthreads();
        // 3. depth = distance to the root, by pointer jumping (9 rounds cover 511 nodes)
        const int nn = 2 * m - 1, root = 2 * m - 2;
        for (int k = t; k < nn; k += kCbBlock) {
            dep[k] = (k == root) ? 0 : 1;
            anc[k] = par[k];
        }
        __syncthreads();
        for (int round = 0; round < 9; ++round) {
            int16_t nd[2], na[2];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int k = t + j * kCbBlock;
                if (k < nn) {
                    nd[j] = (int16_t)(dep[k] + dep[anc[k]]);
                    na[j] = anc[anc[k]];
                }
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int k = t + j * kCbBlock;
                if (k < nn) {
                    dep[k] = nd[j];
                    anc[k] = na[j];
                }
            }
            __syncthreads();
        }
        if (t < m) {
            const int d = dep[t];
            len_s[leaf_sym[t]] = (uint8_t)(d > 255 ? 255 : d);
            atomicMax(&s_max, d);
        }
    } else if (m == 1 && present) {
        len_s[t] = 1;  // one distinct byte: the 1-bit code "0"
        s_max = 1;
    }
    __syncthreads();

    // 4. length limit, then canonical codes
    const int max_len = s_max;
    if (max_len > (int)kMaxCodeLen) {
        set_status(status, HUFF_ERR_CODE_TOO_LONG);
        cb->len[t] = 0;
        cb->code[t] = 0;
        if (t == 0) {
            cb->nsym = 0;
            cb->max_len = 0;
        }
        return;
    }
    const int L = len_s[t];
    if (L)
        atomicAdd(&bl[L], 1u);
    __syncthreads();
    if (t == 0) {
        uint32_t code = 0;
        next_code[0] = 0;
        for (int bits = 1; bits <= (int)kMaxCodeLen; ++bits) {
            code = (code + (bits == 1 ? 0u : bl[bits - 1])) << 1;
            next_code[bits] = code;
        }
    }
    __syncthreads();
    uint32_t code = 0;
    if (L) {
        uint32_t r = 0;
        for (int j = 0; j < t; ++j)
            r += (len_s[j] == L);
        code = next_code[L] + r;
    }
    cb->len[t] = (uint8_t)L;
    cb->code[t] = code;
    if (t == 0) {
        cb->nsym = (uint32_t)m;
        cb->max_len = (uint32_t)max_len;
    }
}

}  // namespace

cudaError_t launch_build_codebook(const unsigned long long *d_hist, huff_codebook_t *d_cb,
                                  int32_t *d_status, cudaStream_t s)
{
    k_build_codebook<<<1, kCbBlock, 0, s>>>(d_hist, d_cb, d_status);
    return cudaGetLastError();
}

}  // namespace huff
