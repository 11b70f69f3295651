// Codebook device routine (one CTA of 256 threads per histogram), shared by
// the single-stream kernel (codebook.cu) and the batched kernel (batch.cu).
// See codebook.cu for the method.
#pragma once

#include "huff_internal.cuh"

namespace huff {
namespace cbk {

struct CodebookShared {
    unsigned long long w[256];
    unsigned long long key[256];               // weight * 256 + byte, all ones if absent
    unsigned long long pm[2][512];             // package-merge: the previous and current list
    uint16_t pos[kMaxCodeLen + 1][256];        // package-merge: position of each leaf per list
    int pm_take[kMaxCodeLen + 1];              // package-merge: leaves taken from each list
    unsigned long long nw[511];  // [0,m): leaves by (weight, byte); [m,2m-1): merged
    int16_t par[511];
    int16_t dep[511];
    int16_t anc[511];
    uint8_t leaf_sym[256];
    uint8_t len_s[256];
    uint32_t bl[kMaxCodeLen + 1];
    uint32_t next_code[kMaxCodeLen + 1];
    int s_max;
};

// Code lengths of at most `limit` bits for the m leaves nw[0..m) (sorted by
// (weight, byte)), by package-merge (Larmore & Hirschberg 1990): list 1 =
// the leaves; list i = the leaves merged with the packages (sums of
// consecutive pairs) of list i-1, a leaf before a package of equal weight;
// the first 2m-2 items of list `limit` are taken and each taken package takes
// its two items of the list below.  A leaf's length is the number of lists
// it is taken from, and the leaves taken from a list are a prefix of the
// sorted leaves.  Every merge position is a binary search (one item per
// thread); 2 <= m <= 2^limit.
__device__ __forceinline__ void package_merge(int m, int limit, CodebookShared &sh)
{
    const int t = threadIdx.x;
    int cnt = m;  // items in the previous list
    if (t < m) {
        sh.pm[0][t] = sh.nw[t];
        sh.pos[1][t] = (uint16_t)t;
    }
    __syncthreads();
    for (int i = 2; i <= limit; ++i) {
        const unsigned long long *prev = sh.pm[(i - 2) & 1];
        unsigned long long *cur = sh.pm[(i - 1) & 1];
        const int np = cnt >> 1;
        if (t < m) {  // leaf t goes after the packages lighter than it
            const unsigned long long w = sh.nw[t];
            int lo = 0, hi = np;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (prev[2 * mid] + prev[2 * mid + 1] < w)
                    lo = mid + 1;
                else
                    hi = mid;
            }
            cur[t + lo] = w;
            sh.pos[i][t] = (uint16_t)(t + lo);
        }
        if (t < np) {  // package t goes after the leaves not heavier than it
            const unsigned long long w = prev[2 * t] + prev[2 * t + 1];
            int lo = 0, hi = m;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (sh.nw[mid] <= w)
                    lo = mid + 1;
                else
                    hi = mid;
            }
            cur[t + lo] = w;
        }
        cnt = m + np;
        __syncthreads();
    }
    if (t == 0) {  // walk down from the last list
        int take = 2 * m - 2;
        for (int i = limit; i >= 1; --i) {
            int lo = 0, hi = m;  // leaves among the first `take` items
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if ((int)sh.pos[i][mid] < take)
                    lo = mid + 1;
                else
                    hi = mid;
            }
            sh.pm_take[i] = lo;
            take = 2 * (take - lo);
        }
    }
    __syncthreads();
    if (t < m) {
        int d = 0;
        for (int i = 1; i <= limit; ++i)
            d += t < sh.pm_take[i];
        sh.dep[t] = (int16_t)d;
    }
}

// Build *cb from hist (u64[256]); blockDim.x must be 256.  Huffman codes
// longer than `limit` (1..32) bits: without `limited` that is an error (*cb
// cleared, HUFF_ERR_CODE_TOO_LONG); with it the lengths are recomputed by
// package-merge (the error only if the bytes present exceed 2^limit).
__device__ __forceinline__ void build_codebook(const unsigned long long *__restrict__ hist,
                                               huff_codebook_t *__restrict__ cb, int32_t *status,
                                               CodebookShared &sh, int limit = (int)kMaxCodeLen,
                                               bool limited = false)
{
    if (chain_failed(status))
        return;
    const int t = threadIdx.x;
    const unsigned long long wt = hist[t];
    // (weight, byte) as one key where every weight is below 2^56 (any byte
    // count is)
    const unsigned long long kt = wt ? (wt << 8) | (unsigned long long)t : ~0ull;
    sh.w[t] = wt;
    sh.key[t] = kt;
    sh.len_s[t] = 0;
    if (t <= (int)kMaxCodeLen)
        sh.bl[t] = 0;
    if (t == 0)
        sh.s_max = 0;
    const int present = wt > 0;
    const int m = __syncthreads_count(present);
    const bool huge = __syncthreads_or((wt >> 56) != 0);  // weights the key cannot hold

    // 1. rank of byte t among present bytes, ordered by (weight, byte): the
    //    keys below its own (an absent byte's key is above every other)
    if (present) {
        int rank = 0;
        if (!huge) {
#pragma unroll 8
            for (int j = 0; j < 256; ++j)
                rank += sh.key[j] < kt;
        } else {
            for (int j = 0; j < 256; ++j) {
                const unsigned long long wj = sh.w[j];
                rank += (wj > 0) & ((wj < wt) | ((wj == wt) & (j < t)));
            }
        }
        sh.leaf_sym[rank] = (uint8_t)t;
        sh.nw[rank] = wt;
    }
    __syncthreads();

    if (m >= 2) {
        // 2. two-queue merge
        if (t == 0) {
            // the first two entries of each queue are kept in registers (all
            // ones past a queue's end), so that a take never waits for a
            // shared load: a leaf's weight is loaded two takes before it can
            // be needed, and a merged node's weight usually never is.  A tie
            // takes the leaf (the smaller id).
            constexpr unsigned long long kNone = ~0ull;
            int li = 0, ii = m, ni = m;
            unsigned long long l0 = sh.nw[0], l1 = sh.nw[1], i0 = kNone, i1 = kNone;  // m >= 2
            for (int step = 0; step < m - 1; ++step) {
                int ab[2];
                unsigned long long wab[2];
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    // branch free: both refills are loaded (at in-range
                    // indices) and the take selects
                    const bool lf = l0 <= i0;
                    const unsigned long long nl = sh.nw[li + 2 < 510 ? li + 2 : 510];
                    const unsigned long long nq = sh.nw[ii + 2 < 510 ? ii + 2 : 510];
                    ab[k] = lf ? li : ii;
                    wab[k] = lf ? l0 : i0;
                    const unsigned long long l1n = li + 2 < m ? nl : kNone;
                    const unsigned long long i1n = ii + 2 < ni ? nq : kNone;
                    l0 = lf ? l1 : l0;
                    l1 = lf ? l1n : l1;
                    i0 = lf ? i0 : i1;
                    i1 = lf ? i1 : i1n;
                    li += lf;
                    ii += !lf;
                }
                const unsigned long long w2 = wab[0] + wab[1];
                sh.nw[ni] = w2;
                sh.par[ab[0]] = (int16_t)ni;
                sh.par[ab[1]] = (int16_t)ni;
                // the new node joins the merged queue at ni
                i0 = ii == ni ? w2 : i0;
                i1 = ii + 1 == ni ? w2 : i1;
                ++ni;
            }
            sh.par[2 * m - 2] = (int16_t)(2 * m - 2);  // the root points at itself
        }
        __syncthreads();
        // 3. depth = distance to the root, by pointer jumping (9 rounds cover
        //    511 nodes; done early once every ancestor is the root)
        const int nn = 2 * m - 1, root = 2 * m - 2;
        for (int k = t; k < nn; k += 256) {
            sh.dep[k] = (k == root) ? 0 : 1;
            sh.anc[k] = sh.par[k];
        }
        __syncthreads();
        for (int round = 0; round < 9; ++round) {
            int16_t nd[2], na[2];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int k = t + j * 256;
                if (k < nn) {
                    nd[j] = (int16_t)(sh.dep[k] + sh.dep[sh.anc[k]]);
                    na[j] = sh.anc[sh.anc[k]];
                }
            }
            __syncthreads();
            bool at_root = true;
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int k = t + j * 256;
                if (k < nn) {
                    sh.dep[k] = nd[j];
                    sh.anc[k] = na[j];
                    at_root &= na[j] == root;
                }
            }
            if (__syncthreads_and(at_root))
                break;
        }
        // the Huffman lengths, unless a limit below 32 is exceeded
        if (t < m)
            atomicMax(&sh.s_max, (int)sh.dep[t]);
        __syncthreads();
        if (limited && sh.s_max > limit && (limit >= 9 || m <= (1 << limit))) {
            __syncthreads();
            if (t == 0)
                sh.s_max = 0;
            package_merge(m, limit, sh);
            if (t < m)
                atomicMax(&sh.s_max, (int)sh.dep[t]);
        }
        if (t < m) {
            const int d = sh.dep[t];
            sh.len_s[sh.leaf_sym[t]] = (uint8_t)(d > 255 ? 255 : d);
        }
    } else if (m == 1 && present) {
        sh.len_s[t] = 1;  // one distinct byte: the 1-bit code "0"
        sh.s_max = 1;
    }
    __syncthreads();

    // 4. length limit, then canonical codes
    const int max_len = sh.s_max;
    if (max_len > limit) {
        set_status(status, HUFF_ERR_CODE_TOO_LONG);
        cb->len[t] = 0;
        cb->code[t] = 0;
        if (t == 0) {
            cb->nsym = 0;
            cb->max_len = 0;
        }
        return;
    }
    const int L = sh.len_s[t];
    if (L)
        atomicAdd(&sh.bl[L], 1u);
    __syncthreads();
    if (t == 0) {
        uint32_t code = 0;
        sh.next_code[0] = 0;
        for (int bits = 1; bits <= (int)kMaxCodeLen; ++bits) {
            code = (code + (bits == 1 ? 0u : sh.bl[bits - 1])) << 1;
            sh.next_code[bits] = code;
        }
    }
    __syncthreads();
    uint32_t code = 0;
    if (L) {
        uint32_t r = 0;
        for (int j = 0; j < t; ++j)
            r += (sh.len_s[j] == L);
        code = sh.next_code[L] + r;
    }
    cb->len[t] = (uint8_t)L;
    cb->code[t] = code;
    if (t == 0) {
        cb->nsym = (uint32_t)m;
        cb->max_len = (uint32_t)max_len;
    }
}

}  // namespace cbk
}  // namespace huff
