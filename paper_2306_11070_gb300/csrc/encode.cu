// Encoder: the coding step of the paper's Huffman Method 1 (Section III-A)
// over Method 2's segments, which become chunks of `cs` symbols with stored
// bit offsets.
//
// Design (one pass over the input, n bytes read + payload written):
//  - The bit offset of every 16 KiB unit is known before this kernel starts
//    (offsets.cu: unit histograms or unit counts, then a scan), so no warp
//    ever waits on another.  Each warp encodes whole units by itself in 16
//    steps of 1024 symbols; the loop has no CTA barrier at all.
//  - A step: every lane loads its 32 bytes (two 16-byte loads, issued one
//    step ahead), looks up the 32 table entries and keeps them in registers,
//    sums them (the low 10 bits of a sum of entries are the sum of their
//    lengths), a warp scan of the sums gives every lane its bit position,
//    the lanes pack their codes into the warp's word buffer in shared
//    memory, and the warp writes the whole words with coalesced stores.  The
//    partial last word is carried in a register into the next step.
//  - Packing: two funnel shifts per code into a 64-bit register; every
//    floor(32 / longest) codes at most one word completes, and a plain store
//    writes the last completed word (see pack32 for why every word ends with
//    the right value without atomics); after a warp barrier each lane ORs
//    its last partial word into the next lane's first word.
//  - Code table in shared memory, replicated per lane ([byte][lane]), so
//    the 32 lookups of a warp never collide in a bank.  Entry =
//    (code << (32 - len)) | len for codes up to 22 bits: the funnel shifts
//    take the length from the entry's low 5 bits.  Longer codes (up to 32
//    bits) use split code / length tables, 16 symbols per lane and a 64-bit
//    accumulator.
//  - The word a unit shares with the unit before it is completed by the later
//    unit: it re-codes the last <= 31 bits of its predecessor from the 32
//    input bytes before it, so no warp waits for another's output and the
//    payload needs no clearing pass.
#include "encode_impl.cuh"

namespace huff {
namespace {

using namespace enc;

// One CTA of 16 warps per SM: one copy of the 32 KiB code table per SM; a
// step keeps 32 table entries per lane in registers (~120 per thread), so
// 16 warps are what fit without spills.
constexpr int kEncBlock = 512;
constexpr int kEncWarps = kEncBlock / 32;
// the (code, 2^len) table is the larger of the two table layouts
constexpr int kEncSmemBytes = (kTbl2Words + kEncWarps * kWarpObuf) * 4;

struct EncodeArgs {
    const uint8_t *in;
    uint64_t n;
    const huff_codebook_t *cb;
    const unsigned long long *unit_off;
    uint32_t cs;
    uint8_t *out;
    uint64_t out_cap;
    unsigned long long *out_bytes;
    int32_t *status;
};

__global__ void __launch_bounds__(kEncBlock, 1) k_encode(EncodeArgs a)
{
    extern __shared__ uint4 smem_raw[];
    // [256][32] (code, 2^len) pairs, or 2 x [256][16] for codes over 22 bits
    uint32_t *tbl = reinterpret_cast<uint32_t *>(smem_raw);
    uint32_t *wob = tbl + kTbl2Words + (threadIdx.x >> 5) * kWarpObuf;  // this warp's buffer

    if (chain_failed(a.status))
        return;
    const Job J = make_job(a.in, a.n, a.cs, a.unit_off, a.out, a.out_cap);
    const uint32_t max_len = a.cb->max_len;
    const bool fast = max_len <= (uint32_t)kFastMaxLen;
    if (fast && mad_group(max_len) >= 3)
        return;  // k_encode_mad codes this stream
    const int group = emit_group(max_len);
    if (blockIdx.x == 0)
        write_header(J, a.cb, a.out_bytes, a.status);
    build_table(a.cb, tbl, fast);
    __syncthreads();  // the only CTA barrier: the table is ready

    const uint64_t nwarps = (uint64_t)gridDim.x * kEncWarps;
    bool overflow = false;
    for (uint64_t u = (uint64_t)blockIdx.x * kEncWarps + (threadIdx.x >> 5); u < J.units; u += nwarps)
        overflow |= encode_unit(J, u, tbl, fast, group, wob);
    if (overflow)
        set_status(a.status, HUFF_ERR_CAPACITY);
}

// The same for codes of at most 10 bits, gathered by multiply-add (see
// encode_impl.cuh); the two kernels are launched back to back and the one
// that does not apply returns at once.
__global__ void __launch_bounds__(kEncBlock, 1) k_encode_mad(EncodeArgs a)
{
    extern __shared__ uint4 smem_raw[];
    uint32_t *tbl2 = reinterpret_cast<uint32_t *>(smem_raw);  // [256][32] (code, 2^len)
    uint32_t *wob = tbl2 + kTbl2Words + (threadIdx.x >> 5) * kWarpObuf;

    if (chain_failed(a.status))
        return;
    const uint32_t max_len = a.cb->max_len;
    const int mgroup = mad_group(max_len);
    if (!(max_len <= (uint32_t)kFastMaxLen && mgroup >= 3))
        return;
    const Job J = make_job(a.in, a.n, a.cs, a.unit_off, a.out, a.out_cap);
    if (blockIdx.x == 0)
        write_header(J, a.cb, a.out_bytes, a.status);
    build_table2(a.cb, tbl2);
    __syncthreads();
    const uint64_t nwarps = (uint64_t)gridDim.x * kEncWarps;
    bool overflow = false;
    for (uint64_t u = (uint64_t)blockIdx.x * kEncWarps + (threadIdx.x >> 5); u < J.units; u += nwarps)
        overflow |= encode_unit_mad_g(J, u, tbl2, mgroup, wob);
    if (overflow)
        set_status(a.status, HUFF_ERR_CAPACITY);
}

}  // namespace

uint64_t encode_workspace_bytes(uint64_t n)
{
    // unit bit counts (u32), unit offsets (u64, + total), the scan's tile sums
    const uint64_t units = (n + kUnitSymbols - 1) / kUnitSymbols;
    return ((4 * units + 255) & ~255ull) + ((8 * (units + 1) + 255) & ~255ull) +
           8 * unit_scan_tiles(units);
}

cudaError_t launch_encode(const uint8_t *d_in, uint64_t n, const huff_codebook_t *d_cb, uint32_t cs,
                          uint8_t *d_out, uint64_t out_cap, unsigned long long *d_out_bytes,
                          void *d_ws, const uint16_t *d_unit_hist, int32_t *d_status,
                          cudaStream_t s)
{
    static KernelSetup setup, setup_mad;
    int per_sm = 0, per_sm_mad = 0;
    cudaError_t err = kernel_setup(setup, (const void *)k_encode, kEncBlock, kEncSmemBytes, &per_sm);
    if (err == cudaSuccess)
        err = kernel_setup(setup_mad, (const void *)k_encode_mad, kEncBlock, kEncSmemBytes, &per_sm_mad);
    if (err != cudaSuccess)
        return err;
    const int sms = device_sm_count();
    if (sms < 1)
        return cudaErrorInvalidDevice;
    const uint64_t units = (n + kUnitSymbols - 1) / kUnitSymbols;
    uint8_t *ws = static_cast<uint8_t *>(d_ws);
    uint32_t *unit_bits = reinterpret_cast<uint32_t *>(ws);
    unsigned long long *unit_off =
        reinterpret_cast<unsigned long long *>(ws + ((4 * units + 255) & ~255ull));
    unsigned long long *tile_sum = reinterpret_cast<unsigned long long *>(
        ws + ((4 * units + 255) & ~255ull) + ((8 * (units + 1) + 255) & ~255ull));
    err = launch_unit_offsets(d_in, n, d_unit_hist, d_cb, unit_bits, unit_off, tile_sum, d_status,
                              s);
    if (err != cudaSuccess)
        return err;
    EncodeArgs a;
    a.in = d_in;
    a.n = n;
    a.cb = d_cb;
    a.unit_off = unit_off;
    a.cs = cs;
    a.out = d_out;
    a.out_cap = out_cap;
    a.out_bytes = d_out_bytes;
    a.status = d_status;
    uint64_t grid = (uint64_t)sms * per_sm;
    const uint64_t want = (units + kEncWarps - 1) / kEncWarps;
    if (grid > want)
        grid = want;
    if (grid < 1)
        grid = 1;
    k_encode_mad<<<(unsigned)grid, kEncBlock, kEncSmemBytes, s>>>(a);
    k_encode<<<(unsigned)grid, kEncBlock, kEncSmemBytes, s>>>(a);
    return cudaGetLastError();
}

}  // namespace huff
