// huff_encode_noalloc: the encoder with its scratch in a fixed, file-scope
// device array instead of a caller workspace.
//
// Some callers cannot allocate device memory when they encode: code running
// between the capture points of a latency-critical loop where an allocation
// would synchronise the device, services that run from a fixed memory
// budget carved out at start-up, and embedding layers that hand the library
// only input and output buffers.  For them the encoder's scratch (the bit
// count and the bit offset of every 16 KiB unit) lives in the array below,
// sized for HUFF_NOALLOC_MAX_SYMBOLS input bytes.  Every GPU that loads this
// library holds it (about 0.75 MiB) until the process exits.
//
// In host code the array's name is only a host-side stand-in; its device
// address is fetched once per device with cudaGetSymbolAddress, on the first
// call made with that device current, and reused afterwards.  All calls share
// the one array: each call writes every scratch entry it reads, so nothing
// needs clearing between calls, but two calls that overlap on the GPU race
// on it.
#include <mutex>

#include "api_trace.h"
#include "huff_internal.cuh"

namespace {

constexpr uint64_t kMaxSymbols = HUFF_NOALLOC_MAX_SYMBOLS;
constexpr uint64_t kMaxUnits = (kMaxSymbols + huff::kUnitSymbols - 1) / huff::kUnitSymbols;
// unit bit counts (u32, padded to 256 bytes), unit offsets (u64, + total,
// padded), the unit scan's tile sums: the encoder's workspace layout
constexpr uint64_t kScratchBytes = ((4 * kMaxUnits + 255) & ~255ull) +
                                   ((8 * (kMaxUnits + 1) + 255) & ~255ull) +
                                   8 * huff::unit_scan_tiles(kMaxUnits);

static __device__ __align__(256) unsigned char g_encode_scratch[kScratchBytes];

std::mutex g_setup_mutex;
void *g_scratch_ptr[huff::kMaxDevices] = {};

// Device address of the scratch array for the current device (set up once).
huff_status_t scratch_address(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return HUFF_ERR_CUDA;
    if (dev < 0 || dev >= huff::kMaxDevices)
        return HUFF_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_encode_scratch) != cudaSuccess || !p)
            return HUFF_ERR_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return HUFF_OK;
}

inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" huff_status_t huff_encode_noalloc(const uint8_t *d_in, uint64_t n,
                                             const huff_codebook_t *d_cb, uint32_t chunk_symbols,
                                             uint8_t *d_out, uint64_t out_cap,
                                             uint64_t *d_out_bytes, int32_t *d_status,
                                             huff_stream_t stream)
{
    HUFF_API_RANGE("huff_encode_noalloc");
    if (!huff::chunk_symbols_valid(chunk_symbols) || !d_cb || !d_out || !d_out_bytes ||
        !d_status || (n && !d_in) || (d_in && !aligned16(d_in)) || !aligned16(d_out))
        return HUFF_ERR_INVALID_ARG;
    if (n > kMaxSymbols || huff::encode_workspace_bytes(n) > kScratchBytes)
        return HUFF_ERR_BUDGET;
    void *ws = nullptr;
    const huff_status_t st = scratch_address(&ws);
    if (st != HUFF_OK)
        return st;
    const cudaError_t err = huff::launch_encode(
        d_in, n, d_cb, chunk_symbols, d_out, out_cap,
        reinterpret_cast<unsigned long long *>(d_out_bytes), ws, nullptr, d_status,
        reinterpret_cast<cudaStream_t>(stream));
    return err == cudaSuccess ? HUFF_OK : HUFF_ERR_CUDA;
}
