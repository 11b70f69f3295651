// C ABI of libhuff: argument checks, workspace layout and kernel launches.
// Every step of the path runs in this library's kernels; nothing here
// touches the data on the host.
#include <cstdint>

#include "api_trace.h"
#include "huff_internal.cuh"

namespace huff {

int current_device()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return -1;
    return dev;
}

int device_sm_count()
{
    static std::atomic<int> cached[kMaxDevices];
    const int dev = current_device();
    if (dev < 0)
        return 0;
    int v = cached[dev].load(std::memory_order_relaxed);
    if (v == 0) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1)
            return 0;
        cached[dev].store(v, std::memory_order_relaxed);
    }
    return v;
}

cudaError_t kernel_setup(KernelSetup &ks, const void *func, int block, size_t dyn_smem,
                         int *per_sm)
{
    const int dev = current_device();
    if (dev < 0)
        return cudaErrorInvalidDevice;
    int v = ks.per_sm[dev].load(std::memory_order_acquire);
    if (v == 0) {
        std::lock_guard<std::mutex> lock(ks.mu);
        v = ks.per_sm[dev].load(std::memory_order_relaxed);
        if (v == 0) {
            cudaError_t err;
            if (dyn_smem > 48 * 1024) {
                err = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)dyn_smem);
                if (err != cudaSuccess)
                    return err;
            }
            err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, func, block, dyn_smem);
            if (err != cudaSuccess)
                return err;
            if (v < 1)
                v = 1;
            ks.per_sm[dev].store(v, std::memory_order_release);
        }
    }
    *per_sm = v;
    return cudaSuccess;
}

namespace {

// huff_compress workspace: histogram, codebook, per-unit histograms, then
// the encoder's part (unit bit counts and offsets).
constexpr uint64_t kWsHistOffset = 0;
constexpr uint64_t kWsCodebookOffset = 2048;
constexpr uint64_t kWsUnitHistOffset = 4096;

inline uint64_t unit_hist_bytes(uint64_t n)
{
    return 512 * ((n + kUnitSymbols - 1) / kUnitSymbols);
}

inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

inline huff_status_t cuda_status(cudaError_t e) { return e == cudaSuccess ? HUFF_OK : HUFF_ERR_CUDA; }

}  // namespace
}  // namespace huff

using namespace huff;

extern "C" {

const char *huff_status_str(huff_status_t status)
{
    switch (status) {
    case HUFF_OK:
        return "ok";
    case HUFF_ERR_INVALID_ARG:
        return "invalid argument";
    case HUFF_ERR_CODE_TOO_LONG:
        return "a code would be longer than 32 bits";
    case HUFF_ERR_CAPACITY:
        return "output buffer too small";
    case HUFF_ERR_CORRUPT_STREAM:
        return "corrupt stream";
    case HUFF_ERR_CUDA:
        return "CUDA error";
    case HUFF_ERR_TIMEOUT:
        return "device wait timed out";
    case HUFF_ERR_BUDGET:
        return "request exceeds the memory budget";
    case HUFF_ERR_UNSUPPORTED:
        return "unsupported";
    default:
        return "unknown status";
    }
}

int huff_version(void) { return 100; }

uint64_t huff_max_stream_size(uint64_t n, uint32_t chunk_symbols)
{
    if (!chunk_symbols_valid(chunk_symbols))
        return 0;
    return kHeaderBytes + 8 * ceil_div_u64(n, chunk_symbols) + 4 * ceil_div_u64(n, 4) + 4;
}

uint64_t huff_workspace_size(uint64_t n, uint32_t chunk_symbols)
{
    if (!chunk_symbols_valid(chunk_symbols))
        return 0;
    const uint64_t b = kWsUnitHistOffset + unit_hist_bytes(n) + encode_workspace_bytes(n);
    return (b + 255) & ~uint64_t(255);
}

huff_status_t huff_histogram(const uint8_t *d_in, uint64_t n, uint64_t *d_hist, huff_stream_t stream)
{
    HUFF_API_RANGE("huff_histogram");
    if (!d_hist || (n && !d_in) || (d_in && !aligned16(d_in)))
        return HUFF_ERR_INVALID_ARG;
    return cuda_status(launch_histogram(d_in, n, reinterpret_cast<unsigned long long *>(d_hist),
                                        nullptr, reinterpret_cast<cudaStream_t>(stream)));
}

uint64_t huff_unit_hist_size(uint64_t n) { return unit_hist_bytes(n); }

huff_status_t huff_histogram_units(const uint8_t *d_in, uint64_t n, uint64_t *d_hist,
                                   uint16_t *d_unit_hist, huff_stream_t stream)
{
    HUFF_API_RANGE("huff_histogram_units");
    if (!d_hist || !d_unit_hist || (n && !d_in) || (d_in && !aligned16(d_in)) ||
        !aligned16(d_unit_hist))
        return HUFF_ERR_INVALID_ARG;
    return cuda_status(launch_histogram(d_in, n, reinterpret_cast<unsigned long long *>(d_hist),
                                        d_unit_hist, reinterpret_cast<cudaStream_t>(stream)));
}

huff_status_t huff_build_codebook(const uint64_t *d_hist, huff_codebook_t *d_cb, int32_t *d_status,
                                  huff_stream_t stream)
{
    HUFF_API_RANGE("huff_build_codebook");
    if (!d_hist || !d_cb || !d_status)
        return HUFF_ERR_INVALID_ARG;
    return cuda_status(launch_build_codebook(reinterpret_cast<const unsigned long long *>(d_hist),
                                             d_cb, d_status,
                                             reinterpret_cast<cudaStream_t>(stream)));
}

huff_status_t huff_build_codebook_limited(const uint64_t *d_hist, uint32_t max_len,
                                          huff_codebook_t *d_cb, int32_t *d_status,
                                          huff_stream_t stream)
{
    HUFF_API_RANGE("huff_build_codebook_limited");
    if (!d_hist || !d_cb || !d_status || max_len < 1 || max_len > kMaxCodeLen)
        return HUFF_ERR_INVALID_ARG;
    return cuda_status(launch_build_codebook(reinterpret_cast<const unsigned long long *>(d_hist),
                                             d_cb, d_status,
                                             reinterpret_cast<cudaStream_t>(stream), max_len));
}

huff_status_t huff_encode(const uint8_t *d_in, uint64_t n, const huff_codebook_t *d_cb,
                          uint32_t chunk_symbols, uint8_t *d_out, uint64_t out_cap,
                          uint64_t *d_out_bytes, void *d_ws, uint64_t ws_bytes, int32_t *d_status,
                          huff_stream_t stream)
{
    HUFF_API_RANGE("huff_encode");
    if (!chunk_symbols_valid(chunk_symbols) || !d_cb || !d_out || !d_out_bytes || !d_ws ||
        !d_status || (n && !d_in) || (d_in && !aligned16(d_in)) || !aligned16(d_out) ||
        !aligned16(d_ws) || ws_bytes < encode_workspace_bytes(n) ||
        n > (uint64_t)UINT32_MAX * kUnitSymbols)
        return HUFF_ERR_INVALID_ARG;
    return cuda_status(launch_encode(d_in, n, d_cb, chunk_symbols, d_out, out_cap,
                                     reinterpret_cast<unsigned long long *>(d_out_bytes), d_ws,
                                     nullptr, d_status, reinterpret_cast<cudaStream_t>(stream)));
}

huff_status_t huff_encode_units(const uint8_t *d_in, uint64_t n, const huff_codebook_t *d_cb,
                                const uint16_t *d_unit_hist, uint32_t chunk_symbols,
                                uint8_t *d_out, uint64_t out_cap, uint64_t *d_out_bytes,
                                void *d_ws, uint64_t ws_bytes, int32_t *d_status,
                                huff_stream_t stream)
{
    HUFF_API_RANGE("huff_encode_units");
    if (!chunk_symbols_valid(chunk_symbols) || !d_cb || !d_out || !d_out_bytes || !d_ws ||
        !d_status || !d_unit_hist || !aligned16(d_unit_hist) || (n && !d_in) ||
        (d_in && !aligned16(d_in)) || !aligned16(d_out) || !aligned16(d_ws) ||
        ws_bytes < encode_workspace_bytes(n) || n > (uint64_t)UINT32_MAX * kUnitSymbols)
        return HUFF_ERR_INVALID_ARG;
    return cuda_status(launch_encode(d_in, n, d_cb, chunk_symbols, d_out, out_cap,
                                     reinterpret_cast<unsigned long long *>(d_out_bytes), d_ws,
                                     d_unit_hist, d_status, reinterpret_cast<cudaStream_t>(stream)));
}

huff_status_t huff_decode(const uint8_t *d_stream, uint64_t stream_bytes, uint8_t *d_out,
                          uint64_t out_cap, uint64_t *d_n, int32_t *d_status, huff_stream_t stream)
{
    HUFF_API_RANGE("huff_decode");
    if (!d_stream || !d_n || !d_status || !aligned16(d_stream) || (d_out && !aligned16(d_out)) ||
        (!d_out && out_cap))
        return HUFF_ERR_INVALID_ARG;
    return cuda_status(launch_decode(d_stream, stream_bytes, d_out, out_cap,
                                     reinterpret_cast<unsigned long long *>(d_n), d_status,
                                     reinterpret_cast<cudaStream_t>(stream)));
}

huff_status_t huff_compress(const uint8_t *d_in, uint64_t n, uint32_t chunk_symbols, uint8_t *d_out,
                            uint64_t out_cap, uint64_t *d_out_bytes, void *d_ws, uint64_t ws_bytes,
                            int32_t *d_status, huff_stream_t stream)
{
    HUFF_API_RANGE("huff_compress");
    if (!chunk_symbols_valid(chunk_symbols) || !d_ws || !aligned16(d_ws) || !d_status ||
        !d_out || !d_out_bytes || (n && !d_in) || (d_in && !aligned16(d_in)) ||
        !aligned16(d_out) || ws_bytes < huff_workspace_size(n, chunk_symbols) ||
        n > (uint64_t)UINT32_MAX * kUnitSymbols)
        return HUFF_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    uint8_t *ws = static_cast<uint8_t *>(d_ws);
    unsigned long long *hist = reinterpret_cast<unsigned long long *>(ws + kWsHistOffset);
    huff_codebook_t *cb = reinterpret_cast<huff_codebook_t *>(ws + kWsCodebookOffset);
    uint16_t *unit_hist = reinterpret_cast<uint16_t *>(ws + kWsUnitHistOffset);
    uint8_t *enc_ws = ws + kWsUnitHistOffset + unit_hist_bytes(n);
    if (cudaMemsetAsync(d_status, 0, sizeof(int32_t), s) != cudaSuccess)
        return HUFF_ERR_CUDA;
    if (launch_histogram(d_in, n, hist, unit_hist, s) != cudaSuccess)
        return HUFF_ERR_CUDA;
    if (launch_build_codebook(hist, cb, d_status, s) != cudaSuccess)
        return HUFF_ERR_CUDA;
    return cuda_status(launch_encode(d_in, n, cb, chunk_symbols, d_out, out_cap,
                                     reinterpret_cast<unsigned long long *>(d_out_bytes), enc_ws,
                                     unit_hist, d_status, s));
}

}  // extern "C"
