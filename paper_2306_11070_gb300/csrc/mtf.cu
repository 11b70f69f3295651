// Move-to-front coding per block: the optional second stage of Method 3
// (Section III-A; Burrows and Wheeler 1994, Section 4).  Every block starts
// from the list 0..255; a byte is coded as its position in the list and then
// moved to the front.
//
// Blocks are cut into 1 KiB segments, one thread each, and the list a
// segment starts from is found without running the blocks serially:
//  - forward: the list at the end of a segment is the segment's distinct
//    bytes, latest occurrence first, followed by the rest of the list it
//    started from in their old order.  k_mtf_distinct writes every
//    segment's distinct bytes (a backward scan); k_mtf_lists, one warp per
//    block, chains them into every segment's starting list (256 bytes per
//    segment); k_mtf_encode codes each segment from its own starting list.
//  - inverse: decoding a segment from the identity list gives, for every
//    position, the index of its byte in the real starting list, and the
//    final list as a permutation of the starting one.  k_mtf_decode_rel does
//    that per segment; k_mtf_lists_inv, one warp per block, composes the
//    permutations into every segment's starting list; k_mtf_map replaces
//    each relative byte by the real one.
// A thread's list lives in shared memory as a column ([entry][thread]
// bytes), so a warp's accesses to equal entries never conflict.
#include "api_trace.h"
#include "huff_internal.cuh"

namespace huff {
namespace {

constexpr uint32_t kSeg = 1024;    // bytes per segment
constexpr int kMtfThreads = 128;   // threads (segments) per CTA of the coding kernels
constexpr int kListWarps = 4;      // warps (blocks) per CTA of the chaining kernels

struct Segs {
    uint64_t n;
    uint32_t block;
    uint32_t per_block;  // segments of a whole block
    uint64_t count;      // segments in all
    __host__ __device__ uint64_t start(uint64_t g) const
    {
        return (g / per_block) * block + (g % per_block) * (uint64_t)kSeg;
    }
    // bytes of segment g (0 past the end of a short last block)
    __host__ __device__ uint32_t len(uint64_t g) const
    {
        const uint64_t bs = (g / per_block) * block;
        const uint64_t be = bs + block < n ? bs + block : n;
        const uint64_t s = start(g);
        if (s >= be)
            return 0;
        return (uint32_t)(be - s < kSeg ? be - s : kSeg);
    }
};

Segs make_segs(uint64_t n, uint32_t block)
{
    Segs S;
    S.n = n;
    S.block = block;
    S.per_block = (block + kSeg - 1) / kSeg;
    const uint64_t blocks = (n + block - 1) / block;
    S.count = blocks * S.per_block;
    return S;
}

// the distinct bytes of every segment, latest occurrence first
__global__ void __launch_bounds__(kMtfThreads) k_mtf_distinct(const uint8_t *in, Segs S,
                                                              uint8_t *dist, uint32_t *dcount)
{
    const uint64_t g = (uint64_t)blockIdx.x * kMtfThreads + threadIdx.x;
    if (g >= S.count)
        return;
    const uint8_t *x = in + S.start(g);
    const uint32_t L = S.len(g);
    uint32_t seen[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    uint32_t k = 0;
    uint8_t *d = dist + g * 256;
    for (uint32_t i = L; i-- > 0;) {
        const uint32_t c = x[i];
        const uint32_t bit = 1u << (c & 31);
        uint32_t w = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j)
            w |= (c >> 5) == (uint32_t)j ? seen[j] : 0u;
        if (!(w & bit)) {
#pragma unroll
            for (int j = 0; j < 8; ++j)
                seen[j] |= (c >> 5) == (uint32_t)j ? bit : 0u;
            d[k++] = (uint8_t)c;
        }
    }
    dcount[g] = k;
}

// One warp per block: the list each segment starts from.  L_0 = 0..255;
// L_{j+1} = distinct bytes of segment j, then the other bytes of L_j in
// their order.
__global__ void __launch_bounds__(kListWarps * 32) k_mtf_lists(const uint8_t *dist,
                                                               const uint32_t *dcount, Segs S,
                                                               uint64_t blocks, uint8_t *lists)
{
    __shared__ __align__(16) uint8_t lst[kListWarps][2][256];
    __shared__ uint32_t mask[kListWarps][8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint64_t b = (uint64_t)blockIdx.x * kListWarps + w;
    if (b >= blocks)
        return;
    for (int i = lane; i < 256; i += 32)
        lst[w][0][i] = (uint8_t)i;
    int cur = 0;
    __syncwarp();
    for (uint32_t j = 0; j < S.per_block; ++j) {
        const uint64_t g = b * S.per_block + j;
        // this segment's starting list
        reinterpret_cast<uint2 *>(lists + g * 256)[lane] =
            reinterpret_cast<const uint2 *>(lst[w][cur])[lane];
        if (S.len(g) == 0)
            continue;  // past the end of a short last block
        const uint32_t k = dcount[g];
        const uint8_t *d = dist + g * 256;
        if (lane < 8)
            mask[w][lane] = 0;
        __syncwarp();
        for (uint32_t i = lane; i < k; i += 32) {
            const uint32_t c = d[i];
            atomicOr(&mask[w][c >> 5], 1u << (c & 31));
            lst[w][cur ^ 1][i] = (uint8_t)c;
        }
        __syncwarp();
        // the bytes of L_j not in the segment keep their order after them
        uint32_t keep[8], nk = 0;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const uint32_t c = lst[w][cur][lane * 8 + t];
            keep[t] = ((mask[w][c >> 5] >> (c & 31)) & 1u) ? 256u : c;
            nk += keep[t] < 256u;
        }
        uint32_t x = nk;
#pragma unroll
        for (int s = 1; s < 32; s <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, s);
            if (lane >= s)
                x += y;
        }
        uint32_t pos = k + x - nk;
#pragma unroll
        for (int t = 0; t < 8; ++t)
            if (keep[t] < 256u)
                lst[w][cur ^ 1][pos++] = (uint8_t)keep[t];
        __syncwarp();
        cur ^= 1;
    }
}

// code each segment from its starting list
__global__ void __launch_bounds__(kMtfThreads) k_mtf_encode(const uint8_t *in, Segs S,
                                                            const uint8_t *lists, uint8_t *out)
{
    __shared__ uint8_t col[256 * kMtfThreads];  // [entry][thread]
    const uint64_t g = (uint64_t)blockIdx.x * kMtfThreads + threadIdx.x;
    if (g >= S.count)
        return;
    uint8_t *l = col + threadIdx.x;
    for (int i = 0; i < 256; ++i)
        l[i * kMtfThreads] = lists[g * 256 + i];
    const uint64_t s0 = S.start(g);
    const uint32_t L = S.len(g);
    for (uint32_t i = 0; i < L; ++i) {
        const uint8_t c = in[s0 + i];
        // walk to c, shifting the entries before it back by one
        uint8_t prev = c, e = l[0];
        uint32_t j = 0;
        while (e != c && j < 255) {  // c is in the list: ends by j = 255
            l[j * kMtfThreads] = prev;
            prev = e;
            ++j;
            e = l[j * kMtfThreads];
        }
        l[j * kMtfThreads] = prev;
        l[0] = c;
        out[s0 + i] = (uint8_t)j;
    }
}

// decode each segment from the identity list: relative bytes and the final
// list (as indices into the starting list)
__global__ void __launch_bounds__(kMtfThreads) k_mtf_decode_rel(const uint8_t *in, Segs S,
                                                                uint8_t *rel, uint8_t *fin)
{
    __shared__ uint8_t col[256 * kMtfThreads];
    const uint64_t g = (uint64_t)blockIdx.x * kMtfThreads + threadIdx.x;
    if (g >= S.count)
        return;
    uint8_t *l = col + threadIdx.x;
    for (int i = 0; i < 256; ++i)
        l[i * kMtfThreads] = (uint8_t)i;
    const uint64_t s0 = S.start(g);
    const uint32_t L = S.len(g);
    for (uint32_t i = 0; i < L; ++i) {
        uint32_t j = in[s0 + i];
        const uint8_t c = l[j * kMtfThreads];
        for (; j > 0; --j)
            l[j * kMtfThreads] = l[(j - 1) * kMtfThreads];
        l[0] = c;
        rel[s0 + i] = c;
    }
    for (int i = 0; i < 256; ++i)
        fin[g * 256 + i] = l[i * kMtfThreads];
}

// One warp per block: L_0 = 0..255, L_{j+1}[i] = L_j[F_j[i]].
__global__ void __launch_bounds__(kListWarps * 32) k_mtf_lists_inv(const uint8_t *fin, Segs S,
                                                                   uint64_t blocks, uint8_t *lists)
{
    __shared__ __align__(16) uint8_t lst[kListWarps][2][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint64_t b = (uint64_t)blockIdx.x * kListWarps + w;
    if (b >= blocks)
        return;
    for (int i = lane; i < 256; i += 32)
        lst[w][0][i] = (uint8_t)i;
    int cur = 0;
    __syncwarp();
    for (uint32_t j = 0; j < S.per_block; ++j) {
        const uint64_t g = b * S.per_block + j;
        reinterpret_cast<uint2 *>(lists + g * 256)[lane] =
            reinterpret_cast<const uint2 *>(lst[w][cur])[lane];
        if (S.len(g) == 0)
            continue;
        const uint2 f = reinterpret_cast<const uint2 *>(fin + g * 256)[lane];
        const uint8_t *fb = reinterpret_cast<const uint8_t *>(&f);
#pragma unroll
        for (int t = 0; t < 8; ++t)
            lst[w][cur ^ 1][lane * 8 + t] = lst[w][cur][fb[t]];
        __syncwarp();
        cur ^= 1;
    }
}

// out[p] = starting list of p's segment, at entry rel[p]
__global__ void k_mtf_map(const uint8_t *rel, Segs S, const uint8_t *lists, uint8_t *out)
{
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < S.n;
         p += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t b = p / S.block;
        const uint64_t g = b * S.per_block + (p - b * S.block) / kSeg;
        out[p] = lists[g * 256 + rel[p]];
    }
}

struct MtfWs {
    uint8_t *dist;      // 256 per segment: distinct bytes, or the final lists
    uint32_t *dcount;   // one per segment
    uint8_t *lists;     // 256 per segment: starting lists
    uint8_t *rel;       // n: relative bytes (inverse)
    uint64_t bytes;
};

MtfWs mtf_layout(uint8_t *base, uint64_t n, uint32_t block)
{
    const Segs S = make_segs(n, block);
    MtfWs w;
    uint64_t off = 0;
    auto carve = [&](uint64_t bytes) {
        uint8_t *p = base ? base + off : nullptr;
        off += (bytes + 255) & ~255ull;
        return p;
    };
    w.dist = carve(256 * S.count);
    w.dcount = reinterpret_cast<uint32_t *>(carve(4 * S.count));
    w.lists = carve(256 * S.count);
    w.rel = carve(n);
    w.bytes = off;
    return w;
}

bool mtf_args_ok(uint64_t n, uint32_t block) { return block >= 1 && n <= HUFF_BWT_MAX_N; }

inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

unsigned seg_grid(uint64_t count) { return (unsigned)((count + kMtfThreads - 1) / kMtfThreads); }

}  // namespace
}  // namespace huff

using namespace huff;

extern "C" {

uint64_t huff_mtf_workspace_size(uint64_t n, uint32_t block)
{
    if (!mtf_args_ok(n, block))
        return 0;
    return mtf_layout(nullptr, n, block).bytes;
}

huff_status_t huff_mtf_forward(const uint8_t *d_in, uint64_t n, uint32_t block, uint8_t *d_out,
                               void *d_ws, uint64_t ws_bytes, huff_stream_t stream)
{
    HUFF_API_RANGE("huff_mtf_forward");
    if (!mtf_args_ok(n, block) || (n && (!d_in || !d_out || !d_ws)) ||
        (n && ws_bytes < huff_mtf_workspace_size(n, block)) || (d_ws && !aligned16(d_ws)))
        return HUFF_ERR_INVALID_ARG;
    if (n == 0)
        return HUFF_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const Segs S = make_segs(n, block);
    const uint64_t blocks = (n + block - 1) / block;
    MtfWs w = mtf_layout(static_cast<uint8_t *>(d_ws), n, block);
    k_mtf_distinct<<<seg_grid(S.count), kMtfThreads, 0, s>>>(d_in, S, w.dist, w.dcount);
    k_mtf_lists<<<(unsigned)((blocks + kListWarps - 1) / kListWarps), kListWarps * 32, 0, s>>>(
        w.dist, w.dcount, S, blocks, w.lists);
    k_mtf_encode<<<seg_grid(S.count), kMtfThreads, 0, s>>>(d_in, S, w.lists, d_out);
    return cudaGetLastError() == cudaSuccess ? HUFF_OK : HUFF_ERR_CUDA;
}

huff_status_t huff_mtf_inverse(const uint8_t *d_in, uint64_t n, uint32_t block, uint8_t *d_out,
                               void *d_ws, uint64_t ws_bytes, huff_stream_t stream)
{
    HUFF_API_RANGE("huff_mtf_inverse");
    if (!mtf_args_ok(n, block) || (n && (!d_in || !d_out || !d_ws)) ||
        (n && ws_bytes < huff_mtf_workspace_size(n, block)) || (d_ws && !aligned16(d_ws)))
        return HUFF_ERR_INVALID_ARG;
    if (n == 0)
        return HUFF_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const Segs S = make_segs(n, block);
    const uint64_t blocks = (n + block - 1) / block;
    MtfWs w = mtf_layout(static_cast<uint8_t *>(d_ws), n, block);
    k_mtf_decode_rel<<<seg_grid(S.count), kMtfThreads, 0, s>>>(d_in, S, w.rel, w.dist);
    k_mtf_lists_inv<<<(unsigned)((blocks + kListWarps - 1) / kListWarps), kListWarps * 32, 0, s>>>(
        w.dist, S, blocks, w.lists);
    const uint64_t gmax = (uint64_t)device_sm_count() * 16;
    const uint64_t gg = (n + 255) / 256 < gmax ? (n + 255) / 256 : gmax;
    k_mtf_map<<<(unsigned)gg, 256, 0, s>>>(w.rel, S, w.lists, d_out);
    return cudaGetLastError() == cudaSuccess ? HUFF_OK : HUFF_ERR_CUDA;
}

}  // extern "C"
