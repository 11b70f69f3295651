// Decoder: reverses the coding of the paper's Huffman Method 1 chunk by
// chunk; Method 2's reassembly by segment id becomes "chunk c writes output
// bytes [c*cs, c*cs + m)" (Section III-A).
//
// Every CTA validates the header and builds the canonical decode tables in
// shared memory from the 256 stored lengths:
//  - a 2^12-entry lookup table (the single-stream kernel keeps one copy, the
//    table code supports C interleaved copies, lane l reading copy l mod C);
//    an entry holds the bytes of up to two codes that fit in the
//    12-bit window, their total length and their number, so text decodes
//    ~2.0 symbols per lookup; a byte table beside it holds the length of the
//    first code alone;
//  - per length, the first canonical code and the index of its first symbol,
//    for codes longer than 12 bits (searched by length).
//
// Parallelism inside a chunk comes from self-synchronisation (Huffman codes
// resynchronise after a few codewords when decoding starts at an arbitrary
// bit; Klein & Wiseman 2003, Weissenberger & Schmidt 2018).  A chunk's bit
// range is cut into S sub-segments, S = 1..32 picked on the device from the
// chunk count so that there are enough independent decoders; one thread per
// sub-segment, S consecutive lanes per chunk:
//  1. every sub-segment but the last counts codewords from its cut point up
//     to the first codeword boundary at or past the next cut, remembering
//     which of its first 256 bits started a codeword;
//  2. sub-segment k's true entry point is where k-1 exits; if that bit is one
//     of k's own early boundaries, k's path has already joined the true one
//     and only its count is corrected, otherwise k re-counts from the entry
//     point (a warp loop that settles in order, usually in one step);
//  3. a segmented scan of the counts gives each sub-segment its output
//     offset; the last one takes the rest of the chunk's symbols;
//  4. each sub-segment decodes its symbols again on the true path, checking
//     every code and the chunk's bit limit.
// Counting (1) and decoding (4) run in windows of lookups.  A window far
// from every lane's segment end (64 lookups here, with the output flushed
// after each 32; 32 in the batched kernel) runs with no checks and no
// branch (warp-uniform); the others (12 lookups) check each code.  Per
// lookup the unchecked window does one 4-byte shared-memory load of the table
// entry, two funnel shifts by the entry itself to drop the bits, and two
// funnel shifts by entry >> 8 that push the entry's symbol bytes into a
// 64-bit output queue; every second lookup refills the bit buffer from the
// input ring and stores the queue's oldest word to the lane's output ring.
// A code longer than the table has an all-zero entry, which consumes and
// emits nothing: the lane waits on it until the next window resolves it.
// Between windows each lane tops up its input ring in shared memory with
// 16-byte cp.async copies that bypass L1 (sixteen 16-byte cells per lane
// here, eight in the batched kernel) and
// stores every completed group of its 128-byte output ring (laid out
// [word][lane], so a warp's accesses never share a bank) with one global
// store: 32-byte groups and 256-bit stores where the chunk's output is
// 32-byte aligned (each lane's write a whole sector), else 16-byte groups.
// The ring holds < 32 unflushed bytes, a window's <= 65 and 3 pending.  The next input word is always preloaded, so the ring's
// latency stays off the per-codeword dependency chain.  The decoded codeword
// sequence is exactly the sequential one, so the stream checks are those of
// a sequential decoder.
#include "decode_impl.cuh"

namespace huff {
namespace {

using namespace dec;

// One 16-warp CTA per SM, one copy of the lookup table (four interleaved
// copies measured the same: the random 12-bit indices conflict as often),
// input rings of 16 cells per lane for 64-lookup windows.
constexpr int kDecBlock = 512;
constexpr int kDecWarps = kDecBlock / 32;
constexpr int kDecCopies = 1;
constexpr int kDecCells = 16;
constexpr size_t kDecInBlock = (size_t)kDecCells * 512;  // 8 KiB per warp
// dynamic shared memory: the tables, then (from the next 8 KiB boundary) one
// 8 KiB input block per warp, then one 4 KiB output block per warp
constexpr size_t kDecTables = (sizeof(DecodeShared<kDecCopies>) + 15) & ~size_t(15);
constexpr size_t kDecSmem = kDecTables + kDecInBlock + (size_t)kDecWarps * (kDecInBlock + 4096);

struct DecodeArgs {
    const uint8_t *stream;
    uint64_t bytes;
    uint8_t *out;
    uint64_t cap;
    unsigned long long *d_n;
    int32_t *status;
    uint32_t min_chains;
};

__global__ void __launch_bounds__(kDecBlock, 1) k_decode(DecodeArgs a)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    DecodeShared<kDecCopies> &sh = *reinterpret_cast<DecodeShared<kDecCopies> *>(dsm);
    const uint32_t tbl_end = smem_u32(dsm) + (uint32_t)kDecTables;
    // warps' input blocks, then output blocks
    const uint32_t rings = (tbl_end + (uint32_t)kDecInBlock - 1u) & ~((uint32_t)kDecInBlock - 1u);
    uint16_t *scratch = reinterpret_cast<uint16_t *>(dsm + (rings - smem_u32(dsm)));  // free while tables build

    if (chain_failed(a.status))
        return;
    // CTAs past the last task leave before building tables (block 0 always
    // stays: it reports header errors)
    if (blockIdx.x > 0 && a.bytes >= kHeaderBytes) {
        const uint64_t n = *reinterpret_cast<const uint64_t *>(a.stream + 256);
        const uint32_t cs = *reinterpret_cast<const uint32_t *>(a.stream + 264);
        if (chunk_symbols_valid(cs)) {
            const uint64_t chunks = n / cs + (n % cs != 0);
            const uint32_t S = pick_split(chunks, a.min_chains);
            const uint64_t tasks = (chunks + (32 / S) - 1) / (32 / S);
            if ((uint64_t)blockIdx.x >= tasks)
                return;
        }
    }
    StreamInfo si;
    if (!prepare<kDecBlock>(a.stream, a.bytes, a.out, a.cap, a.d_n, a.status,
                            blockIdx.x == 0 && threadIdx.x == 0, sh, scratch, si, threadIdx.x, CtaSync()))
        return;
    const uint32_t S = pick_split(si.chunks, a.min_chains);
    const uint64_t tasks = (si.chunks + (32 / S) - 1) / (32 / S);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint32_t in_s = rings + wib * (uint32_t)kDecInBlock + lane * 16;
    const uint32_t out_s = rings + kDecWarps * (uint32_t)kDecInBlock + wib * 4096 + lane * 4;
    // tasks are dealt to the CTAs in turn (task t to CTA t mod grid), so
    // when there are fewer tasks than warps every SM still gets its share
    const uint64_t nwarps = (uint64_t)gridDim.x * kDecWarps;
    for (uint64_t task = (uint64_t)wib * gridDim.x + blockIdx.x; task < tasks; task += nwarps) {
        if (decode_task<kDecCells>(si, S, task, in_s, out_s)) {
            if (lane == 0)
                set_status(a.status, HUFF_ERR_CORRUPT_STREAM);
            return;
        }
    }
}

KernelSetup g_decode_setup;

}  // namespace

cudaError_t launch_decode(const uint8_t *d_stream, uint64_t bytes, uint8_t *d_out, uint64_t out_cap,
                          unsigned long long *d_n, int32_t *d_status, cudaStream_t s)
{
    int per_sm = 0;
    cudaError_t err = kernel_setup(g_decode_setup, (const void *)k_decode, kDecBlock, kDecSmem,
                                   &per_sm);
    if (err != cudaSuccess)
        return err;
    const int sms = device_sm_count();
    if (sms < 1)
        return cudaErrorInvalidDevice;
    // the chunk count is only known on the device; bound it by the table size
    const uint64_t max_chunks = bytes > kHeaderBytes ? (bytes - kHeaderBytes) / 8 : 0;
    uint64_t grid = (max_chunks + kDecWarps - 1) / kDecWarps;
    const uint64_t cap = (uint64_t)sms * per_sm;
    if (grid > cap)
        grid = cap;
    if (grid < 1)
        grid = 1;
    DecodeArgs a;
    a.stream = d_stream;
    a.bytes = bytes;
    a.out = d_out;
    a.cap = out_cap;
    a.d_n = d_n;
    a.status = d_status;
    a.min_chains = (uint32_t)sms * 256u;
    k_decode<<<(unsigned)grid, kDecBlock, kDecSmem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace huff
