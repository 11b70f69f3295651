// Segmented container: one codebook per segment, the paper's Method 2 taken
// literally (Section III-A: segments with ids, each coded with its own tree,
// reassembled by id).  Layout in huff.h.
//
// Compression runs the batched engine over the segments into worst-case
// slots of the caller's workspace (so no segment waits on another's size),
// then k_seg_finish lays out the container header and start table from the
// actual stream sizes and k_seg_gather moves every stream to its place
// (16-byte copies, zero padding).  Decompression reads the header and start
// table on the host, validates them, and runs the batched decoder with every
// segment's stream and output range; k_seg_check turns the per-segment
// results into one status.
#include <cstring>
#include <vector>

#include "api_trace.h"
#include "huff_internal.cuh"

namespace huff {
namespace {

constexpr int kSegBlock = 256;

__host__ __device__ inline uint64_t al16(uint64_t v) { return (v + 15) & ~15ull; }
inline uint64_t al256(uint64_t v) { return (v + 255) & ~255ull; }

struct SegLayout {
    uint64_t count, last, slot, header, slots_bytes, sizes_off, status_off, ws_bytes;
};

bool seg_layout(uint64_t n, uint64_t seg, uint32_t cs, SegLayout &L)
{
    if (seg < 16 || (seg & 15) || !chunk_symbols_valid(cs))
        return false;
    L.count = n ? (n + seg - 1) / seg : 0;
    L.last = n ? n - (L.count - 1) * seg : 0;
    L.slot = al16(huff_max_stream_size(seg < n ? seg : n, cs));
    L.header = al16(24 + 8 * (L.count + 1));
    L.slots_bytes = L.count * L.slot;
    L.sizes_off = al256(L.slots_bytes);
    L.status_off = al256(L.sizes_off + 8 * L.count);
    L.ws_bytes = al256(L.status_off + 4 * L.count) + 256;
    return true;
}

// Header, start table and container size from the actual stream sizes; the
// first segment error (or a capacity error) into *status.
__global__ void __launch_bounds__(kSegBlock)
    k_seg_finish(const uint64_t *__restrict__ sizes, const int32_t *__restrict__ sts,
                 uint64_t count, uint64_t n, uint64_t seg, uint64_t header, uint8_t *out,
                 uint64_t out_cap, uint64_t *out_bytes, int32_t *status)
{
    __shared__ unsigned long long s_warp[kSegBlock / 32];
    __shared__ unsigned long long s_total;
    __shared__ int s_err;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0)
        s_err = 0;
    __syncthreads();
    uint64_t *hdr = reinterpret_cast<uint64_t *>(out);
    unsigned long long carry = header;
    for (uint64_t t0 = 0; t0 < count; t0 += kSegBlock) {
        const uint64_t i = t0 + tid;
        const unsigned long long own = i < count ? al16(sizes[i]) : 0ull;
        if (i < count && sts[i] != 0)
            atomicCAS(&s_err, 0, sts[i]);
        unsigned long long x = own;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d)
                x += y;
        }
        if (lane == 31)
            s_warp[warp] = x;
        __syncthreads();
        if (warp == 0) {
            const unsigned long long w = lane < kSegBlock / 32 ? s_warp[lane] : 0ull;
            unsigned long long z = w;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, z, d);
                if (lane >= d)
                    z += y;
            }
            if (lane < kSegBlock / 32)
                s_warp[lane] = z - w;
            if (lane == 31)
                s_total = z;
        }
        __syncthreads();
        if (i < count)
            hdr[3 + i] = carry + s_warp[warp] + x - own;  // start[i]
        carry += s_total;
        __syncthreads();
    }
    if (tid == 0) {
        hdr[0] = n;
        hdr[1] = seg;
        hdr[2] = count;
        hdr[3 + count] = carry;  // the container size
        *out_bytes = carry;
        if (s_err)
            set_status(status, s_err);
        else if (carry > out_cap)
            set_status(status, HUFF_ERR_CAPACITY);
    }
    // zero the gap between the table and start[0]
    for (uint64_t b = 24 + 8 * (count + 1) + tid; b < header; b += kSegBlock)
        out[b] = 0;
}

// Move segment streams from their slots to their places, zero padded to 16.
__global__ void __launch_bounds__(kSegBlock)
    k_seg_gather(const uint8_t *__restrict__ slots, uint64_t slot, const uint64_t *__restrict__ sizes,
                 uint64_t count, uint8_t *out, const int32_t *status)
{
    if (chain_failed(status))
        return;
    const uint64_t *start = reinterpret_cast<const uint64_t *>(out) + 3;
    for (uint64_t i = blockIdx.x; i < count; i += gridDim.x) {
        const uint64_t size = sizes[i], nv = (size + 15) >> 4;
        const uint4 *src = reinterpret_cast<const uint4 *>(slots + i * slot);
        uint4 *dst = reinterpret_cast<uint4 *>(out + start[i]);
        for (uint64_t v = threadIdx.x; v < nv; v += kSegBlock) {
            uint4 q = src[v];
            const uint64_t keep = size - 16 * v;  // bytes of this vector inside the stream
            if (keep < 16) {
                uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint64_t lo = 4 * (uint64_t)k;
                    if (keep <= lo)
                        w[k] = 0u;
                    else if (keep < lo + 4)
                        w[k] &= 0xffffffffu >> (8 * (lo + 4 - keep));
                }
                q = make_uint4(w[0], w[1], w[2], w[3]);
            }
            dst[v] = q;
        }
    }
}

// Per-segment results of a container decode into one status.
__global__ void __launch_bounds__(kSegBlock)
    k_seg_check(const uint64_t *__restrict__ got_n, const int32_t *__restrict__ sts,
                uint64_t count, uint64_t n, uint64_t seg, int32_t *status)
{
    for (uint64_t i = threadIdx.x; i < count; i += kSegBlock) {
        const uint64_t want = i + 1 < count ? seg : n - (count - 1) * seg;
        if (sts[i] != 0)
            set_status(status, sts[i] == HUFF_ERR_CAPACITY ? HUFF_ERR_CORRUPT_STREAM : sts[i]);
        else if (got_n[i] != want)
            set_status(status, HUFF_ERR_CORRUPT_STREAM);
    }
}

huff_status_t put_status(int32_t *d_status, int32_t v, cudaStream_t s)
{
    static const int32_t vals[] = {HUFF_ERR_CORRUPT_STREAM, HUFF_ERR_CAPACITY};
    const int32_t *src = v == HUFF_ERR_CORRUPT_STREAM ? &vals[0] : &vals[1];
    if (cudaMemcpyAsync(d_status, src, sizeof(int32_t), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return HUFF_ERR_CUDA;
    return HUFF_OK;
}

inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace
}  // namespace huff

using namespace huff;

extern "C" {

uint64_t huff_segmented_max_size(uint64_t n, uint64_t segment_bytes, uint32_t chunk_symbols)
{
    SegLayout L;
    if (!seg_layout(n, segment_bytes, chunk_symbols, L))
        return 0;
    uint64_t total = L.header;
    for (uint64_t i = 0; i < L.count; ++i)
        total += al16(huff_max_stream_size(i + 1 < L.count ? segment_bytes : L.last, chunk_symbols));
    return total;
}

uint64_t huff_segmented_workspace_size(uint64_t n, uint64_t segment_bytes, uint32_t chunk_symbols)
{
    SegLayout L;
    return seg_layout(n, segment_bytes, chunk_symbols, L) ? L.ws_bytes : 0;
}

huff_status_t huff_segmented_compress(const uint8_t *d_in, uint64_t n, uint64_t segment_bytes,
                                      uint32_t chunk_symbols, uint8_t *d_out, uint64_t out_cap,
                                      uint64_t *d_out_bytes, void *d_ws, uint64_t ws_bytes,
                                      int32_t *d_status, huff_stream_t stream)
{
    HUFF_API_RANGE("huff_segmented_compress");
    SegLayout L;
    if (!seg_layout(n, segment_bytes, chunk_symbols, L) || !d_out || !d_out_bytes || !d_status ||
        (n && !d_in) || !d_ws || ws_bytes < L.ws_bytes || out_cap < L.header ||
        (d_in && !aligned16(d_in)) || !aligned16(d_out) || !aligned16(d_ws))
        return HUFF_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    uint8_t *ws = static_cast<uint8_t *>(d_ws);
    uint64_t *sizes = reinterpret_cast<uint64_t *>(ws + L.sizes_off);
    int32_t *sts = reinterpret_cast<int32_t *>(ws + L.status_off);
    if (cudaMemsetAsync(d_status, 0, sizeof(int32_t), s) != cudaSuccess)
        return HUFF_ERR_CUDA;
    if (L.count) {
        std::vector<huff_batch_desc_t> descs(L.count);
        for (uint64_t i = 0; i < L.count; ++i) {
            descs[i].d_in = d_in + i * segment_bytes;
            descs[i].in_bytes = i + 1 < L.count ? segment_bytes : L.last;
            descs[i].d_out = ws + i * L.slot;
            descs[i].out_cap = L.slot;
            descs[i].d_out_bytes = sizes + i;
            descs[i].d_status = sts + i;
        }
        huff_batch_params_t prm;
        huff_batch_default_params(&prm);
        prm.chunk_symbols = chunk_symbols;
        prm.use_graph = 0;  // one run
        huff_batch_plan_t *plan = nullptr;
        if (L.count > 0xffffffffull)
            return HUFF_ERR_INVALID_ARG;
        huff_status_t st = huff_batch_plan(descs.data(), (uint32_t)L.count, HUFF_BATCH_COMPRESS,
                                           &prm, &plan);
        if (st == HUFF_OK)
            st = huff_batch_run(plan, stream);
        if (st == HUFF_OK && cudaStreamSynchronize(s) != cudaSuccess)
            st = HUFF_ERR_CUDA;
        huff_batch_destroy(plan);
        if (st != HUFF_OK)
            return st;
    }
    k_seg_finish<<<1, kSegBlock, 0, s>>>(sizes, sts, L.count, n, segment_bytes, L.header, d_out,
                                         out_cap, d_out_bytes, d_status);
    if (cudaGetLastError() != cudaSuccess)
        return HUFF_ERR_CUDA;
    if (L.count) {
        const uint64_t grid = L.count < (uint64_t)device_sm_count() * 8 ? L.count
                                                                         : (uint64_t)device_sm_count() * 8;
        k_seg_gather<<<(unsigned)grid, kSegBlock, 0, s>>>(ws, L.slot, sizes, L.count, d_out, d_status);
        if (cudaGetLastError() != cudaSuccess)
            return HUFF_ERR_CUDA;
    }
    return HUFF_OK;
}

huff_status_t huff_segmented_decompress(const uint8_t *d_in, uint64_t in_bytes, uint8_t *d_out,
                                        uint64_t out_cap, uint64_t *d_n, int32_t *d_status,
                                        huff_stream_t stream)
{
    HUFF_API_RANGE("huff_segmented_decompress");
    if (!d_in || !d_n || !d_status || !aligned16(d_in) || (out_cap && !d_out))
        return HUFF_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(d_status, 0, sizeof(int32_t), s) != cudaSuccess)
        return HUFF_ERR_CUDA;
    if (in_bytes < 32)
        return put_status(d_status, HUFF_ERR_CORRUPT_STREAM, s);
    uint64_t h[3];
    if (cudaMemcpyAsync(h, d_in, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return HUFF_ERR_CUDA;
    const uint64_t n = h[0], seg = h[1], count = h[2];
    if (seg < 16 || (seg & 15) || count != (n ? (n + seg - 1) / seg : 0) ||
        count > (in_bytes - 32) / 8)
        return put_status(d_status, HUFF_ERR_CORRUPT_STREAM, s);
    std::vector<uint64_t> start(count + 1);
    if (cudaMemcpyAsync(start.data(), d_in + 24, 8 * (count + 1), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return HUFF_ERR_CUDA;
    const uint64_t header = al16(24 + 8 * (count + 1));
    bool ok = start[0] == header && start[count] <= in_bytes;
    for (uint64_t i = 0; i < count && ok; ++i)
        ok = (start[i] & 15) == 0 && start[i + 1] >= start[i];
    if (!ok)
        return put_status(d_status, HUFF_ERR_CORRUPT_STREAM, s);
    if (cudaMemcpyAsync(d_n, &n, sizeof(uint64_t), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return HUFF_ERR_CUDA;
    if (n > out_cap)
        return put_status(d_status, HUFF_ERR_CAPACITY, s);
    if (count == 0)
        return HUFF_OK;
    if (count > 0xffffffffull)
        return put_status(d_status, HUFF_ERR_CORRUPT_STREAM, s);
    if (!aligned16(d_out))
        return HUFF_ERR_INVALID_ARG;
    uint8_t *scratch = nullptr;
    if (cudaMalloc(&scratch, 12 * count + 16) != cudaSuccess)
        return HUFF_ERR_CUDA;
    uint64_t *got = reinterpret_cast<uint64_t *>(scratch);
    int32_t *sts = reinterpret_cast<int32_t *>(scratch + 8 * count);
    std::vector<huff_batch_desc_t> descs(count);
    for (uint64_t i = 0; i < count; ++i) {
        descs[i].d_in = d_in + start[i];
        descs[i].in_bytes = start[i + 1] - start[i];
        descs[i].d_out = d_out + i * seg;
        descs[i].out_cap = i + 1 < count ? seg : n - (count - 1) * seg;
        descs[i].d_out_bytes = got + i;
        descs[i].d_status = sts + i;
    }
    huff_batch_params_t prm;
    huff_batch_default_params(&prm);
    prm.use_graph = 0;
    // spread each segment over enough lanes that the whole container fills
    // about one wave of decoders (256 lanes per SM, the single-stream rule)
    {
        const uint64_t want = ((uint64_t)device_sm_count() * 256 + count - 1) / count;
        uint32_t lanes = 32;
        while (lanes < want && lanes < 65536)
            lanes <<= 1;
        prm.decode_lanes = lanes;
    }
    huff_batch_plan_t *plan = nullptr;
    huff_status_t st = huff_batch_plan(descs.data(), (uint32_t)count, HUFF_BATCH_DECOMPRESS, &prm,
                                       &plan);
    if (st == HUFF_ERR_INVALID_ARG) {  // descriptors taken from a malformed table
        cudaFree(scratch);
        return put_status(d_status, HUFF_ERR_CORRUPT_STREAM, s);
    }
    if (st == HUFF_OK)
        st = huff_batch_run(plan, stream);
    if (st == HUFF_OK) {
        k_seg_check<<<1, kSegBlock, 0, s>>>(got, sts, count, n, seg, d_status);
        if (cudaGetLastError() != cudaSuccess)
            st = HUFF_ERR_CUDA;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess && st == HUFF_OK)
        st = HUFF_ERR_CUDA;
    huff_batch_destroy(plan);
    cudaFree(scratch);
    return st;
}

}  // extern "C"
