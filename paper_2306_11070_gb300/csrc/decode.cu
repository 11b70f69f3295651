// Decoder: reverses the coding of the paper's Huffman Method 1 chunk by
// chunk; Method 2's reassembly by segment id becomes "chunk c writes output
// bytes [c*cs, c*cs + m)" (Section III-A).
//
// Every CTA validates the header and builds the canonical decode tables in
// shared memory from the 256 stored lengths: a 2^11-entry lookup table for
// codes of up to 11 bits (entry = byte | length << 8) and, per length, the
// first code and the index of its first symbol for longer codes.  One thread
// decodes one chunk from its stored bit offset with a 64-bit bit buffer fed
// by aligned 32-bit loads, and writes 16 output bytes at a time.
#include "huff_internal.cuh"

namespace huff {
namespace {

constexpr int kDecBlock = 128;
constexpr int kLutBits = 11;

__global__ void __launch_bounds__(kDecBlock)
    k_decode(const uint8_t *__restrict__ stream, uint64_t bytes, uint8_t *__restrict__ out,
             uint64_t cap, unsigned long long *d_n, int32_t *status)
{
    __shared__ uint16_t lut[1 << kLutBits];
    __shared__ uint8_t len_s[256];
    __shared__ uint8_t sorted[256];
    __shared__ uint32_t count[kMaxCodeLen + 1];
    __shared__ uint32_t first[kMaxCodeLen + 1];
    __shared__ uint32_t start[kMaxCodeLen + 1];
    __shared__ unsigned long long s_kraft;
    __shared__ int s_max, s_nsym, s_bad;

    if (chain_failed(status))
        return;
    const int tid = threadIdx.x;
    const bool reporter = blockIdx.x == 0 && tid == 0;
    if (bytes < kHeaderBytes) {
        if (reporter)
            set_status(status, HUFF_ERR_CORRUPT_STREAM);
        return;
    }
    const uint64_t n = *reinterpret_cast<const uint64_t *>(stream + 256);
    const uint32_t cs = *reinterpret_cast<const uint32_t *>(stream + 264);
    const uint32_t max_field = *reinterpret_cast<const uint32_t *>(stream + 268);
    if (!chunk_symbols_valid(cs)) {
        if (reporter)
            set_status(status, HUFF_ERR_CORRUPT_STREAM);
        return;
    }
    const uint64_t chunks = n / cs + (n % cs != 0);
    if (chunks > (bytes - kHeaderBytes) / 8) {
        if (reporter)
            set_status(status, HUFF_ERR_CORRUPT_STREAM);
        return;
    }

    // ---- lengths: range, longest, count, Kraft sum ----
    if (tid <= (int)kMaxCodeLen)
        count[tid] = 0;
    if (tid == 0) {
        s_kraft = 0;
        s_max = 0;
        s_nsym = 0;
        s_bad = 0;
    }
    __syncthreads();
    for (int b = tid; b < 256; b += kDecBlock) {
        const uint32_t L = stream[b];
        len_s[b] = (uint8_t)L;
        if (L > kMaxCodeLen) {
            s_bad = 1;
        } else if (L) {
            atomicMax(&s_max, (int)L);
            atomicAdd(&s_nsym, 1);
            atomicAdd(&s_kraft, 1ull << (32 - L));
            atomicAdd(&count[L], 1u);
        }
    }
    __syncthreads();
    const uint32_t max_len = (uint32_t)s_max;
    const int nsym = s_nsym;
    bool bad = s_bad || max_len != max_field || (n > 0 && nsym == 0) ||
               (nsym == 1 && max_len != 1) || (nsym >= 2 && s_kraft != (1ull << 32));
    if (bad) {
        if (reporter)
            set_status(status, HUFF_ERR_CORRUPT_STREAM);
        return;
    }
    if (reporter)
        *d_n = n;
    if (n > cap) {
        if (reporter)
            set_status(status, HUFF_ERR_CAPACITY);
        return;
    }
    if (n == 0)
        return;

    // ---- canonical tables (RFC 1951 next_code recurrence) ----
    if (tid == 0) {
        uint32_t code = 0, idx = 0;
        for (uint32_t L = 1; L <= kMaxCodeLen; ++L) {
            code = (code + count[L - 1]) << 1;
            first[L] = code;
            start[L] = idx;
            idx += count[L];
        }
    }
    __syncthreads();
    for (int b = tid; b < 256; b += kDecBlock) {
        const uint32_t L = len_s[b];
        if (L) {
            uint32_t r = 0;
            for (int j = 0; j < b; ++j)
                r += len_s[j] == L;
            sorted[start[L] + r] = (uint8_t)b;
        }
    }
    __syncthreads();
    const uint32_t lut_len = max_len < (uint32_t)kLutBits ? max_len : (uint32_t)kLutBits;
    for (int v = tid; v < (1 << kLutBits); v += kDecBlock) {
        uint16_t ent = 0;
        for (uint32_t L = 1; L <= lut_len; ++L) {
            const uint32_t c = (uint32_t)v >> (kLutBits - L);
            if (count[L] && c - first[L] < count[L]) {
                ent = (uint16_t)(sorted[start[L] + c - first[L]] | (L << 8));
                break;
            }
        }
        lut[v] = ent;
    }
    __syncthreads();

    const uint64_t pay_words = (bytes - kHeaderBytes - 8 * chunks) / 4;
    const uint64_t pbits = 32 * pay_words;
    const uint64_t *offs = reinterpret_cast<const uint64_t *>(stream + kHeaderBytes);
    const uint32_t *pay = reinterpret_cast<const uint32_t *>(stream + kHeaderBytes + 8 * chunks);

    for (uint64_t c = (uint64_t)blockIdx.x * kDecBlock + tid; c < chunks;
         c += (uint64_t)gridDim.x * kDecBlock) {
        uint64_t pos = offs[c];
        const uint64_t limit = c + 1 < chunks ? offs[c + 1] : pbits;
        if ((c == 0 && pos != 0) || pos > limit) {
            set_status(status, HUFF_ERR_CORRUPT_STREAM);
            return;
        }
        const uint64_t obase = c * cs;
        const uint64_t m = n - obase < cs ? n - obase : cs;

        // bit buffer: valid bits left-aligned in buf, `have` of them
        uint64_t wi = pos >> 5;
        uint64_t buf = (uint64_t)(wi < pay_words ? pay[wi] : 0u) << 32;
        buf <<= (pos & 31);
        int have = 32 - (int)(pos & 31);
        ++wi;
        bool ok = true;

        auto next_symbol = [&]() -> uint32_t {
            if (have <= 32) {
                buf |= (uint64_t)(wi < pay_words ? pay[wi] : 0u) << (32 - have);
                have += 32;
                ++wi;
            }
            const uint32_t ent = lut[buf >> (64 - kLutBits)];
            uint32_t L = ent >> 8, sym = ent & 0xffu;
            if (L == 0) {  // longer than the table: canonical search by length
                const uint32_t v = (uint32_t)(buf >> 32);
                for (L = lut_len + 1; L <= max_len; ++L) {
                    const uint32_t cv = v >> (32 - L);
                    if (count[L] && cv - first[L] < count[L]) {
                        sym = sorted[start[L] + cv - first[L]];
                        break;
                    }
                }
                if (L > max_len) {
                    ok = false;
                    L = 1;
                }
            }
            if (pos + L > limit)
                ok = false;
            pos += L;
            buf <<= L;
            have -= (int)L;
            return sym;
        };

        uint64_t i = 0;
        for (; i + 16 <= m && ok; i += 16) {
            uint32_t q[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int k = 0; k < 16; ++k)
                q[k >> 2] |= next_symbol() << (8 * (k & 3));
            *reinterpret_cast<uint4 *>(out + obase + i) = make_uint4(q[0], q[1], q[2], q[3]);
        }
        for (; i < m && ok; ++i)
            out[obase + i] = (uint8_t)next_symbol();
        if (!ok || (c + 1 < chunks && pos != limit)) {
            set_status(status, HUFF_ERR_CORRUPT_STREAM);
            return;
        }
    }
}

}  // namespace

cudaError_t launch_decode(const uint8_t *d_stream, uint64_t bytes, uint8_t *d_out, uint64_t out_cap,
                          unsigned long long *d_n, int32_t *d_status, cudaStream_t s)
{
    static int per_sm = 0;
    cudaError_t err;
    if (per_sm == 0) {
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_decode, kDecBlock, 0);
        if (err != cudaSuccess)
            return err;
        if (per_sm < 1)
            per_sm = 1;
    }
    // the chunk count is only known on the device; bound it by the table size
    const uint64_t max_chunks = bytes > kHeaderBytes ? (bytes - kHeaderBytes) / 8 : 0;
    uint64_t grid = (max_chunks + kDecBlock - 1) / kDecBlock;
    const uint64_t cap = (uint64_t)device_sm_count() * per_sm;
    if (grid > cap)
        grid = cap;
    if (grid < 1)
        grid = 1;
    k_decode<<<(unsigned)grid, kDecBlock, 0, s>>>(d_stream, bytes, d_out, out_cap, d_n, d_status);
    return cudaGetLastError();
}

}  // namespace huff
