// Autotuner of the batched engine (huff_batch_autotune in huff.h).
//
// The best launch parameters of the fused batch kernels depend on the shape
// of the batch: how many lanes a buffer's chunks are spread over
// (decode_lanes; small buffers need sub-chunk splitting to fill a warp, big
// ones do not), how many persistent CTAs share an SM, and the chunk size the
// streams are written with (smaller chunks give a small buffer more
// independent decoders at the cost of a larger offset table).  The tuner
// plans the caller's own batch with each candidate, times a few runs with
// CUDA events on the caller's stream and keeps the fastest; the result is
// cached per (device, operation, batch shape).  With HUFF_TUNE_CACHE set to
// a file path the cache also persists there, one JSON object per line
// (device name and SM count, operation, shape, chosen parameters): read on
// the first call, a line appended for every newly tuned shape.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "api_trace.h"
#include "huff_internal.cuh"

namespace {

struct ShapeKey {
    std::string device;  // name and SM count
    int op;
    uint32_t count_log2, total_log2, mean_log2, cs, round_trip;
    bool operator<(const ShapeKey &o) const
    {
        return std::tie(device, op, count_log2, total_log2, mean_log2, cs, round_trip) <
               std::tie(o.device, o.op, o.count_log2, o.total_log2, o.mean_log2, o.cs,
                        o.round_trip);
    }
};

std::mutex g_mu;
std::map<ShapeKey, huff_batch_params_t> g_cache;
bool g_file_read = false;

const char *cache_path()
{
    const char *p = std::getenv("HUFF_TUNE_CACHE");
    return p && *p ? p : nullptr;
}

// entries of the cache file (g_mu held); lines that do not parse are skipped
void read_cache_file()
{
    g_file_read = true;
    const char *path = cache_path();
    if (!path)
        return;
    FILE *f = std::fopen(path, "r");
    if (!f)
        return;
    char line[512];
    while (std::fgets(line, sizeof line, f)) {
        char dev[200];
        ShapeKey k;
        huff_batch_params_t p;
        huff_batch_default_params(&p);
        unsigned op, c, t, m, cs, rt, chunk, ctas, lanes;
        if (std::sscanf(line,
                        "{\"device\": \"%199[^\"]\", \"op\": %u, \"count_log2\": %u, "
                        "\"total_log2\": %u, \"mean_log2\": %u, \"cs\": %u, \"round_trip\": %u, "
                        "\"chunk_symbols\": %u, \"ctas_per_sm\": %u, \"decode_lanes\": %u}",
                        dev, &op, &c, &t, &m, &cs, &rt, &chunk, &ctas, &lanes) != 10)
            continue;
        const bool lanes_ok = lanes >= 1 && lanes <= 256 && (lanes & (lanes - 1)) == 0;
        if (!huff::chunk_symbols_valid(chunk) || !lanes_ok || ctas > 64 || rt > 1 ||
            (op != HUFF_BATCH_COMPRESS && op != HUFF_BATCH_DECOMPRESS))
            continue;  // not a set the tuner could have chosen
        k.device = dev;
        k.op = (int)op;
        k.count_log2 = c;
        k.total_log2 = t;
        k.mean_log2 = m;
        k.cs = cs;
        k.round_trip = rt;
        p.chunk_symbols = chunk;
        p.ctas_per_sm = ctas;
        p.decode_lanes = lanes;
        g_cache[k] = p;
    }
    std::fclose(f);
}

// append one entry (g_mu held)
void append_cache_file(const ShapeKey &k, const huff_batch_params_t &p)
{
    const char *path = cache_path();
    if (!path)
        return;
    FILE *f = std::fopen(path, "a");
    if (!f)
        return;
    std::fprintf(f,
                 "{\"device\": \"%s\", \"op\": %d, \"count_log2\": %u, \"total_log2\": %u, "
                 "\"mean_log2\": %u, \"cs\": %u, \"round_trip\": %u, \"chunk_symbols\": %u, "
                 "\"ctas_per_sm\": %u, \"decode_lanes\": %u}\n",
                 k.device.c_str(), k.op, k.count_log2, k.total_log2, k.mean_log2, k.cs,
                 k.round_trip, p.chunk_symbols, p.ctas_per_sm, p.decode_lanes);
    std::fclose(f);
}

std::string device_id(int device)
{
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess)
        return std::to_string(device);
    std::string name(prop.name);
    for (char &ch : name)
        if (ch == '"' || ch == '\\' || ch == '\n')
            ch = ' ';
    return name + "/" + std::to_string(prop.multiProcessorCount);
}

uint32_t log2_bucket(double v) { return v < 1.0 ? 0u : (uint32_t)std::floor(std::log2(v)); }

// Mean time of `reps` runs of plan p (after one warm-up run), in ms.
huff_status_t time_plan(huff_batch_plan_t *p, cudaStream_t s, int reps, float &ms)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0)
            cudaEventDestroy(e0);
        return HUFF_ERR_CUDA;
    }
    huff_status_t st = huff_batch_run(p, reinterpret_cast<huff_stream_t>(s));
    if (st == HUFF_OK && cudaEventRecord(e0, s) != cudaSuccess)
        st = HUFF_ERR_CUDA;
    for (int r = 0; r < reps && st == HUFF_OK; ++r)
        st = huff_batch_run(p, reinterpret_cast<huff_stream_t>(s));
    if (st == HUFF_OK && (cudaEventRecord(e1, s) != cudaSuccess ||
                          cudaEventSynchronize(e1) != cudaSuccess ||
                          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        st = HUFF_ERR_CUDA;
    if (st == HUFF_OK)
        ms /= (float)reps;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

// Plan + time one parameter set.
huff_status_t try_params(const huff_batch_desc_t *descs, uint32_t count, huff_op_t op,
                         const huff_batch_params_t &prm, cudaStream_t s, float &ms)
{
    huff_batch_plan_t *p = nullptr;
    huff_status_t st = huff_batch_plan(descs, count, op, &prm, &p);
    if (st == HUFF_OK)
        st = time_plan(p, s, 3, ms);
    huff_batch_destroy(p);
    return st;
}

const uint32_t kLanes[] = {32, 64, 128, 256};
const uint32_t kCtas[] = {0, 1};

// Best decompress parameters of a batch of streams; base supplies the rest.
huff_status_t tune_decompress(const huff_batch_desc_t *descs, uint32_t count,
                              const huff_batch_params_t &base, cudaStream_t s,
                              huff_batch_params_t &best, float &best_ms)
{
    best_ms = -1.0f;
    for (uint32_t lanes : kLanes)
        for (uint32_t ctas : kCtas) {
            huff_batch_params_t prm = base;
            prm.decode_lanes = lanes;
            prm.ctas_per_sm = ctas;
            float ms = 0.0f;
            const huff_status_t st = try_params(descs, count, HUFF_BATCH_DECOMPRESS, prm, s, ms);
            if (st != HUFF_OK)
                return st;
            if (best_ms < 0.0f || ms < best_ms) {
                best_ms = ms;
                best = prm;
            }
        }
    return HUFF_OK;
}

}  // namespace

extern "C" huff_status_t huff_batch_autotune(const huff_batch_desc_t *descs, uint32_t count,
                                             huff_op_t op, const huff_batch_params_t *base,
                                             uint32_t flags, huff_batch_params_t *best,
                                             huff_stream_t stream)
{
    HUFF_API_RANGE("huff_batch_autotune");
    if (!descs || count == 0 || !best ||
        (op != HUFF_BATCH_COMPRESS && op != HUFF_BATCH_DECOMPRESS))
        return HUFF_ERR_INVALID_ARG;
    huff_batch_params_t b0;
    huff_batch_default_params(&b0);
    if (base)
        b0 = *base;
    b0.barrier_extra = 0;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const bool round_trip = op == HUFF_BATCH_COMPRESS && (flags & HUFF_TUNE_ROUND_TRIP);

    double total = 0.0;
    for (uint32_t i = 0; i < count; ++i)
        total += (double)descs[i].in_bytes;
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess)
        return HUFF_ERR_CUDA;
    const ShapeKey key{device_id(device), (int)op, log2_bucket(count), log2_bucket(total),
                       log2_bucket(total / count), b0.chunk_symbols, round_trip ? 1u : 0u};
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_file_read)
            read_cache_file();
        if (!(flags & HUFF_TUNE_FORCE)) {
            auto it = g_cache.find(key);
            if (it != g_cache.end()) {
                // tuned fields from the cache, the rest from base
                *best = b0;
                best->chunk_symbols = it->second.chunk_symbols;
                best->ctas_per_sm = it->second.ctas_per_sm;
                best->decode_lanes = it->second.decode_lanes;
                return HUFF_OK;
            }
        }
    }

    huff_batch_params_t chosen = b0;
    huff_status_t st = HUFF_OK;
    if (op == HUFF_BATCH_DECOMPRESS) {
        float ms = 0.0f;
        st = tune_decompress(descs, count, b0, s, chosen, ms);
    } else {
        // a chunk size is a candidate only if every stream surely fits
        std::vector<uint32_t> sizes{b0.chunk_symbols};
        bool fits = b0.chunk_symbols != 4096u;
        for (uint32_t i = 0; i < count && fits; ++i)
            fits = descs[i].out_cap >= huff_max_stream_size(descs[i].in_bytes, 4096u);
        if (fits)
            sizes.push_back(4096u);
        // decoded-byte scratch for the round trip, and per-buffer results
        uint8_t *scratch = nullptr;
        uint64_t *d_n = nullptr;
        int32_t *d_st = nullptr;
        std::vector<huff_batch_desc_t> dd;
        if (round_trip) {
            std::vector<uint64_t> off(count + 1, 0);
            for (uint32_t i = 0; i < count; ++i)
                off[i + 1] = off[i] + ((descs[i].in_bytes + 15) & ~15ull) + 16;
            if (cudaMalloc(&scratch, off[count] ? off[count] : 16) != cudaSuccess ||
                cudaMalloc(&d_n, sizeof(uint64_t) * count) != cudaSuccess ||
                cudaMalloc(&d_st, sizeof(int32_t) * count) != cudaSuccess)
                st = HUFF_ERR_CUDA;
            dd.resize(count);
            for (uint32_t i = 0; i < count && st == HUFF_OK; ++i) {
                dd[i].d_in = descs[i].d_out;  // the stream just written (trailing bytes ignored)
                dd[i].in_bytes = descs[i].out_cap;
                dd[i].d_out = scratch + off[i];
                dd[i].out_cap = descs[i].in_bytes;
                dd[i].d_out_bytes = d_n + i;
                dd[i].d_status = d_st + i;
            }
        }
        float best_score = -1.0f;
        for (size_t k = 0; k < sizes.size() && st == HUFF_OK; ++k) {
            huff_batch_params_t prm = b0;
            prm.chunk_symbols = sizes[k];
            float ms_c = 0.0f;
            // compress with every CTA count, keep the faster
            huff_batch_params_t best_c = prm;
            float best_c_ms = -1.0f;
            for (uint32_t ctas : kCtas) {
                huff_batch_params_t q = prm;
                q.ctas_per_sm = ctas;
                st = try_params(descs, count, HUFF_BATCH_COMPRESS, q, s, ms_c);
                if (st != HUFF_OK)
                    break;
                if (best_c_ms < 0.0f || ms_c < best_c_ms) {
                    best_c_ms = ms_c;
                    best_c = q;
                }
            }
            if (st != HUFF_OK)
                break;
            float score = best_c_ms;
            huff_batch_params_t cand = best_c;
            if (round_trip) {
                // the outputs now hold streams of the last timed run: re-run
                // the best compress setting so they are that setting's streams
                huff_batch_plan_t *p = nullptr;
                st = huff_batch_plan(descs, count, HUFF_BATCH_COMPRESS, &best_c, &p);
                if (st == HUFF_OK)
                    st = huff_batch_run(p, stream);
                if (st == HUFF_OK && cudaStreamSynchronize(s) != cudaSuccess)
                    st = HUFF_ERR_CUDA;
                huff_batch_destroy(p);
                huff_batch_params_t dbest;
                float ms_d = 0.0f;
                if (st == HUFF_OK)
                    st = tune_decompress(dd.data(), count, best_c, s, dbest, ms_d);
                if (st != HUFF_OK)
                    break;
                score += ms_d;
                cand.decode_lanes = dbest.decode_lanes;
            }
            if (best_score < 0.0f || score < best_score) {
                best_score = score;
                chosen = cand;
            }
        }
        if (round_trip && st == HUFF_OK) {
            // leave the caller's outputs holding streams of the chosen setting
            huff_batch_plan_t *p = nullptr;
            st = huff_batch_plan(descs, count, HUFF_BATCH_COMPRESS, &chosen, &p);
            if (st == HUFF_OK)
                st = huff_batch_run(p, stream);
            if (st == HUFF_OK && cudaStreamSynchronize(s) != cudaSuccess)
                st = HUFF_ERR_CUDA;
            huff_batch_destroy(p);
        }
        cudaFree(scratch);
        cudaFree(d_n);
        cudaFree(d_st);
    }
    if (st != HUFF_OK)
        return st;
    chosen.use_graph = b0.use_graph;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_cache[key] = chosen;
        append_cache_file(key, chosen);
    }
    *best = chosen;
    return HUFF_OK;
}
