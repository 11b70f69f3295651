// Served path: a request loop with continuous batching.
//
// Clients submit compress or decompress requests (host buffers) at any time.
// A scheduler thread admits waiting requests, in arrival order per
// operation, into the next round as soon as a round slot (a CUDA stream) is
// free and the device arena -- the memory budget, reserved once -- has room
// for their inputs, outputs and the round's scratch.  A round copies its
// inputs in, runs the fused batch kernel (one cooperative launch over all its
// requests, each with its own codebook; batch.cu) and copies back the sizes
// and statuses, then exactly the result bytes.  Several rounds are in flight
// at once on different streams, each on a share of the SMs, so requests that
// arrive while others run start as soon as a slot and memory free up, and
// their work overlaps on the device.  A request's result never depends on
// what else is in its round: every buffer is coded on its own.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "api_trace.h"
#include "batch_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;
using huff::BatchLayout;

constexpr uint64_t kAlign = 256;
inline uint64_t align_up(uint64_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// First-fit allocator of offsets inside the device arena.
class Arena {
  public:
    void init(uint64_t cap)
    {
        free_.clear();
        if (cap)
            free_[0] = cap;
    }
    bool alloc(uint64_t size, uint64_t &off)
    {
        size = align_up(size ? size : 1);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= size) {
                off = it->first;
                const uint64_t rest = it->second - size;
                free_.erase(it);
                if (rest)
                    free_[off + size] = rest;
                return true;
            }
        }
        return false;
    }
    void release(uint64_t off, uint64_t size)
    {
        size = align_up(size ? size : 1);
        auto it = free_.emplace(off, size).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }

  private:
    std::map<uint64_t, uint64_t> free_;
};

struct Req {
    uint64_t ticket;
    int32_t op;
    const uint8_t *h_in;
    uint64_t in_bytes;
    uint8_t *h_out;
    uint64_t out_cap;
    uint64_t need_out;  // device output bytes
    uint64_t off_in, off_out;
    double t_submit, t_start, t_done;
    int32_t status;
    uint64_t out_bytes;
    int32_t done;
};

struct Round {
    huff_op_t op;
    cudaStream_t s;
    cudaEvent_t ev_kernel, ev_copy;
    int stage;  // 0 idle, 1 kernel + size readback in flight, 2 result copies in flight
    std::vector<Req *> reqs;
    uint64_t off_block, block_bytes;  // batch block + sizes/status words in the arena
    uint8_t *h_stage;                 // pinned: descriptors upload and size readback
    uint64_t h_stage_bytes;
};

}  // namespace

struct huff_server {
    huff_server_cfg_t cfg;
    int device;
    uint8_t *d_arena;
    Arena arena;
    std::vector<Round> rounds;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req *> pending;
    std::unordered_map<uint64_t, Req *> reqs;
    std::thread loop;
    std::atomic<bool> stop;
    uint64_t next_ticket;
    Clock::time_point t0;
    unsigned grid;
    int rr;  // which operation gets the next free slot first
};

namespace {

double now_s(const huff_server_t *S)
{
    return std::chrono::duration<double>(Clock::now() - S->t0).count();
}

uint64_t out_need(const huff_server_t *S, int32_t op, uint64_t in_bytes, uint64_t out_cap)
{
    return op == HUFF_BATCH_COMPRESS ? huff_max_stream_size(in_bytes, S->cfg.chunk_symbols)
                                     : out_cap;
}

// Device block bytes of a round over `count` requests of `units` total.
uint64_t round_block_bytes(uint32_t count, uint64_t units)
{
    // descriptors and prefixes; per unit its histogram, offset and owner; per
    // encode item (at most units / 8 + count) its owner; codebooks
    return 4096 + 64ull * count + 16ull * (count + 1) * 3 + 536ull * units + 16ull * count +
           16ull * (units / huff::kUnitsPerItem + count) + 512 + sizeof(huff_codebook_t) * count;
}

// Try to start a round of `op` on slot r; returns true if it launched.
bool start_round(huff_server_t *S, Round &r, huff_op_t op)
{
    std::vector<Req *> take;
    uint64_t units = 0;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        bool blocked = false;
        for (auto it = S->pending.begin(); it != S->pending.end() && !blocked;) {
            Req *q = *it;
            if (q->op != (int32_t)op) {
                ++it;
                continue;
            }
            if (take.size() >= S->cfg.max_batch)
                break;
            uint64_t oi = 0, oo = 0;
            const bool a1 = S->arena.alloc(q->in_bytes, oi);
            const bool a2 = a1 && S->arena.alloc(q->need_out, oo);
            if (!a2) {
                if (a1)
                    S->arena.release(oi, q->in_bytes);
                blocked = true;  // arrival order: later requests wait behind it
                break;
            }
            q->off_in = oi;
            q->off_out = oo;
            take.push_back(q);
            units += op == HUFF_BATCH_COMPRESS ? (q->in_bytes + huff::kUnitSymbols - 1) /
                                                     huff::kUnitSymbols
                                               : 0;
            it = S->pending.erase(it);
        }
        if (take.empty())
            return false;
        // the round's scratch; if it does not fit, hand the requests back
        r.block_bytes = round_block_bytes((uint32_t)take.size(), units);
        if (!S->arena.alloc(r.block_bytes, r.off_block)) {
            for (auto rit = take.rbegin(); rit != take.rend(); ++rit) {
                S->arena.release((*rit)->off_in, (*rit)->in_bytes);
                S->arena.release((*rit)->off_out, (*rit)->need_out);
                S->pending.push_front(*rit);
            }
            return false;
        }
        const double t = now_s(S);
        for (Req *q : take)
            q->t_start = t;
    }
    r.op = op;
    r.reqs = take;
    const uint32_t count = (uint32_t)take.size();
    uint8_t *blk = S->d_arena + r.off_block;
    // sizes and statuses live at the end of the block
    uint8_t *d_meta = blk + r.block_bytes - 16ull * count;
    std::vector<huff_batch_desc_t> descs(count);
    for (uint32_t i = 0; i < count; ++i) {
        Req *q = take[i];
        descs[i].d_in = S->d_arena + q->off_in;
        descs[i].in_bytes = q->in_bytes;
        descs[i].d_out = S->d_arena + q->off_out;
        descs[i].out_cap = q->need_out;
        descs[i].d_out_bytes = reinterpret_cast<uint64_t *>(d_meta + 8ull * i);
        descs[i].d_status = reinterpret_cast<int32_t *>(d_meta + 8ull * count + 4ull * i);
    }
    BatchLayout L;
    huff::batch_layout(descs.data(), count, op, L);
    bool ok = L.bytes + 16ull * count <= r.block_bytes && L.upload_bytes <= r.h_stage_bytes &&
              16ull * count <= r.h_stage_bytes;
    for (uint32_t i = 0; ok && i < count; ++i)
        ok = cudaMemcpyAsync(const_cast<uint8_t *>(descs[i].d_in), take[i]->h_in,
                             take[i]->in_bytes, cudaMemcpyHostToDevice, r.s) == cudaSuccess;
    ok = ok && huff::batch_upload(L, blk, r.h_stage, r.s) == cudaSuccess;
    if (ok) {
        // a decompress round of few requests spreads each over more lanes,
        // so that the round alone fills about one wave of decoders
        uint32_t lanes = S->cfg.decode_lanes;
        if (op == HUFF_BATCH_DECOMPRESS) {
            const uint64_t want = ((uint64_t)huff::device_sm_count() * 256 + count - 1) / count;
            while (lanes < want && lanes < 65536)
                lanes <<= 1;
        }
        const huff::BatchArgs args = huff::batch_args(L, blk, S->cfg.chunk_symbols, lanes);
        ok = huff::batch_launch(op, args, S->grid, r.s) == cudaSuccess;
    }
    ok = ok && cudaMemcpyAsync(r.h_stage, d_meta, 16ull * count, cudaMemcpyDeviceToHost, r.s) ==
                   cudaSuccess;
    ok = ok && cudaEventRecord(r.ev_kernel, r.s) == cudaSuccess;
    if (!ok) {
        cudaStreamSynchronize(r.s);
        std::lock_guard<std::mutex> lk(S->mu);
        const double t = now_s(S);
        for (Req *q : take) {
            q->status = HUFF_ERR_CUDA;
            q->t_done = t;
            q->done = 1;
            S->arena.release(q->off_in, q->in_bytes);
            S->arena.release(q->off_out, q->need_out);
        }
        S->arena.release(r.off_block, r.block_bytes);
        r.reqs.clear();
        S->cv_done.notify_all();
        return false;
    }
    r.stage = 1;
    return true;
}

// Advance round r if its work finished; returns true on progress.
bool poll_round(huff_server_t *S, Round &r)
{
    if (r.stage == 1 && cudaEventQuery(r.ev_kernel) == cudaSuccess) {
        const uint32_t count = (uint32_t)r.reqs.size();
        const uint64_t *sizes = reinterpret_cast<const uint64_t *>(r.h_stage);
        const int32_t *sts = reinterpret_cast<const int32_t *>(r.h_stage + 8ull * count);
        for (uint32_t i = 0; i < count; ++i) {
            Req *q = r.reqs[i];
            q->status = sts[i];
            q->out_bytes = sizes[i];
            if (q->status == HUFF_OK && q->out_bytes > q->out_cap)
                q->status = HUFF_ERR_CAPACITY;
            if (q->status == HUFF_OK && q->out_bytes)
                cudaMemcpyAsync(q->h_out, S->d_arena + q->off_out, q->out_bytes,
                                cudaMemcpyDeviceToHost, r.s);
        }
        cudaEventRecord(r.ev_copy, r.s);
        r.stage = 2;
        return true;
    }
    if (r.stage == 2 && cudaEventQuery(r.ev_copy) == cudaSuccess) {
        std::lock_guard<std::mutex> lk(S->mu);
        const double t = now_s(S);
        for (Req *q : r.reqs) {
            q->t_done = t;
            q->done = 1;
            S->arena.release(q->off_in, q->in_bytes);
            S->arena.release(q->off_out, q->need_out);
        }
        S->arena.release(r.off_block, r.block_bytes);
        r.reqs.clear();
        r.stage = 0;
        S->cv_done.notify_all();
        return true;
    }
    return false;
}

void server_loop(huff_server_t *S)
{
    cudaSetDevice(S->device);
    for (;;) {
        bool progress = false;
        for (Round &r : S->rounds)
            progress |= poll_round(S, r);
        bool busy = false;
        for (Round &r : S->rounds)
            busy |= r.stage != 0;
        if (S->stop.load() && !busy) {
            std::lock_guard<std::mutex> lk(S->mu);
            if (S->pending.empty())
                break;
        }
        for (Round &r : S->rounds) {
            if (r.stage != 0)
                continue;
            const huff_op_t first = S->rr ? HUFF_BATCH_DECOMPRESS : HUFF_BATCH_COMPRESS;
            const huff_op_t second = S->rr ? HUFF_BATCH_COMPRESS : HUFF_BATCH_DECOMPRESS;
            if (start_round(S, r, first) || start_round(S, r, second)) {
                S->rr ^= 1;
                progress = true;
            }
        }
        if (!progress) {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait_for(lk, std::chrono::microseconds(20));
        }
    }
}

void destroy_server(huff_server_t *S)
{
    if (!S)
        return;
    if (S->loop.joinable()) {
        S->stop.store(true);
        S->cv_work.notify_all();
        S->loop.join();
    }
    for (Round &r : S->rounds) {
        if (r.s) {
            cudaStreamSynchronize(r.s);
            cudaStreamDestroy(r.s);
        }
        if (r.ev_kernel)
            cudaEventDestroy(r.ev_kernel);
        if (r.ev_copy)
            cudaEventDestroy(r.ev_copy);
        if (r.h_stage)
            cudaFreeHost(r.h_stage);
    }
    for (auto &kv : S->reqs)  // every request, pending or not, is in this map
        delete kv.second;
    if (S->d_arena)
        cudaFree(S->d_arena);
    delete S;
}

}  // namespace

extern "C" {

void huff_server_default_config(huff_server_cfg_t *cfg)
{
    if (!cfg)
        return;
    cfg->device_budget = 8ull << 30;
    cfg->max_rounds = 3;
    cfg->max_batch = 256;
    cfg->chunk_symbols = HUFF_DEFAULT_CHUNK_SYMBOLS;
    cfg->decode_lanes = 128;
}

huff_status_t huff_server_create(const huff_server_cfg_t *cfg, huff_server_t **out)
{
    HUFF_API_RANGE("huff_server_create");
    if (!out)
        return HUFF_ERR_INVALID_ARG;
    *out = nullptr;
    huff_server_cfg_t c;
    huff_server_default_config(&c);
    if (cfg)
        c = *cfg;
    if (c.device_budget < (1ull << 20) || c.max_rounds == 0 || c.max_rounds > 16 ||
        c.max_batch == 0 || !huff::chunk_symbols_valid(c.chunk_symbols) || c.decode_lanes == 0 ||
        c.decode_lanes > 65536)
        return HUFF_ERR_INVALID_ARG;
    huff_server_t *S = new (std::nothrow) huff_server_t();
    if (!S)
        return HUFF_ERR_CUDA;
    S->cfg = c;
    S->d_arena = nullptr;
    S->stop.store(false);
    S->next_ticket = 1;
    S->rr = 0;
    S->t0 = Clock::now();
    if (cudaGetDevice(&S->device) != cudaSuccess ||
        cudaMalloc(&S->d_arena, c.device_budget) != cudaSuccess) {
        destroy_server(S);
        return HUFF_ERR_CUDA;
    }
    S->arena.init(c.device_budget);
    // each round gets an equal share of the resident CTAs of the heavier kernel
    const int occ = std::min(huff::batch_occupancy(HUFF_BATCH_COMPRESS),
                             huff::batch_occupancy(HUFF_BATCH_DECOMPRESS));
    if (occ < 1) {
        destroy_server(S);
        return HUFF_ERR_CUDA;
    }
    S->grid = std::max(1u, (unsigned)(huff::device_sm_count() * occ) / c.max_rounds);
    S->rounds.resize(c.max_rounds);
    for (Round &r : S->rounds) {
        r = Round();
        r.h_stage_bytes = 4096 + 128ull * c.max_batch;
        if (cudaStreamCreateWithFlags(&r.s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&r.ev_kernel, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&r.ev_copy, cudaEventDisableTiming) != cudaSuccess ||
            cudaMallocHost(&r.h_stage, r.h_stage_bytes) != cudaSuccess) {
            destroy_server(S);
            return HUFF_ERR_CUDA;
        }
    }
    S->loop = std::thread(server_loop, S);
    *out = S;
    return HUFF_OK;
}

huff_status_t huff_server_submit(huff_server_t *S, const huff_request_t *req, uint64_t *ticket)
{
    HUFF_API_RANGE("huff_server_submit");
    if (!S || !req || !ticket || (req->op != HUFF_BATCH_COMPRESS && req->op != HUFF_BATCH_DECOMPRESS) ||
        (req->in_bytes && !req->h_in) || !req->h_out)
        return HUFF_ERR_INVALID_ARG;
    if (req->op == HUFF_BATCH_DECOMPRESS && req->in_bytes < huff::kHeaderBytes)
        return HUFF_ERR_INVALID_ARG;
    Req *q = new (std::nothrow) Req();
    if (!q)
        return HUFF_ERR_CUDA;
    std::memset(q, 0, sizeof(*q));
    q->op = req->op;
    q->h_in = req->h_in;
    q->in_bytes = req->in_bytes;
    q->h_out = req->h_out;
    q->out_cap = req->out_cap;
    q->need_out = out_need(S, req->op, req->in_bytes, req->out_cap);
    const uint64_t units =
        req->op == HUFF_BATCH_COMPRESS ? (req->in_bytes + huff::kUnitSymbols - 1) / huff::kUnitSymbols : 0;
    const uint64_t need = align_up(q->in_bytes ? q->in_bytes : 1) + align_up(q->need_out) +
                          align_up(round_block_bytes(1, units));
    if (need > S->cfg.device_budget || q->need_out == 0) {
        delete q;
        return HUFF_ERR_BUDGET;  // could never be admitted
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        q->ticket = S->next_ticket++;
        q->t_submit = now_s(S);
        S->reqs[q->ticket] = q;
        S->pending.push_back(q);
        *ticket = q->ticket;
    }
    S->cv_work.notify_one();
    return HUFF_OK;
}

static void fill_result(const Req *q, huff_result_t *res)
{
    res->done = q->done;
    res->status = q->done ? q->status : HUFF_OK;
    res->out_bytes = q->done ? q->out_bytes : 0;
    res->t_submit = q->t_submit;
    res->t_start = q->t_start;
    res->t_done = q->t_done;
}

huff_status_t huff_server_poll(huff_server_t *S, uint64_t ticket, huff_result_t *res)
{
    if (!S || !res)
        return HUFF_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end())
        return HUFF_ERR_INVALID_ARG;
    fill_result(it->second, res);
    return HUFF_OK;
}

huff_status_t huff_server_wait(huff_server_t *S, uint64_t ticket, uint32_t timeout_ms,
                               huff_result_t *res)
{
    HUFF_API_RANGE("huff_server_wait");
    if (!S || !res)
        return HUFF_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end())
        return HUFF_ERR_INVALID_ARG;
    Req *q = it->second;
    const bool done = S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                                          [q] { return q->done != 0; });
    fill_result(q, res);
    return done ? HUFF_OK : HUFF_ERR_TIMEOUT;
}

huff_status_t huff_server_release(huff_server_t *S, uint64_t ticket)
{
    if (!S)
        return HUFF_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end() || !it->second->done)
        return HUFF_ERR_INVALID_ARG;
    delete it->second;
    S->reqs.erase(it);
    return HUFF_OK;
}

void huff_server_destroy(huff_server_t *S) { destroy_server(S); }

}  // extern "C"
