// rr_serve.cu -- continuous batching of planning requests (include/rr.h,
// "serving"). A worker thread admits queued requests as their grid and move
// buffers fit in a device input pool, plans them in waves with
// rr_plan_batched on a pool of
// streams (one context, hence one workspace arena, per stream, so waves run
// concurrently on the device), gives each planned request result memory from
// a device heap once its exact size (16 B per elementary step) is known, and
// batches it in a second wave (RR_BATCH_ONLY). Submitting, polling and
// releasing only touch host-side queues under a mutex.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>
#include "rr_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

enum Phase { QUEUED = 0, PLANNING = 1, PLANNED = 2, BATCHING = 3, DONE = 4 };

struct Req {
    int64_t ticket = 0;
    std::vector<uint8_t> grid;
    int layout = 0, m = 0, n = 0;
    rr_rect rect{0, 0, 0, 0};
    int64_t inOff = -1, inBytes = 0;          // grid + move list in the input pool
    int64_t heapOff = -1, heapBytes = 0;
    int phase = QUEUED;
    rr_instance desc{};
    double tSubmit = 0, tAdmit = 0, tDone = 0;
};

struct Wave {
    bool busy = false;
    int kind = 0;                 // 1 plan, 2 batch
    cudaEvent_t ev = nullptr;
    std::vector<Req *> reqs;
};

// First-fit allocator over [0, size) of the device heap.
struct Heap {
    std::map<int64_t, int64_t> freeList;   // offset -> bytes
    int64_t size = 0;
    void init(int64_t s) { size = s; freeList.clear(); if (s > 0) freeList[0] = s; }
    static int64_t round(int64_t b) { return (b + 255) & ~(int64_t)255; }
    int64_t alloc(int64_t bytes)
    {
        bytes = round(bytes);
        for (auto it = freeList.begin(); it != freeList.end(); ++it) {
            if (it->second >= bytes) {
                const int64_t off = it->first, rest = it->second - bytes;
                freeList.erase(it);
                if (rest) freeList[off + bytes] = rest;
                return off;
            }
        }
        return -1;
    }
    void release(int64_t off, int64_t bytes)
    {
        bytes = round(bytes);
        auto it = freeList.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != freeList.end() && it->first + it->second == nx->first) { it->second += nx->second; freeList.erase(nx); }
        if (it != freeList.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) { pv->second += it->second; freeList.erase(it); }
        }
    }
};

// Room for a request's moves: every atom moves at most twice (an outer
// column's atom once in its column, once to a receiver), and there are at
// most m n atoms.
int64_t moves_cap(int m, int n) { return 2ll * m * n; }

}  // namespace

struct rr_server {
    rr_serve_config cfg{};
    int device = 0;
    int64_t gridBytes = 0;                    // largest grid (staging buffers)
    char *inBase = nullptr;                   // input pool: grids and move lists
    Heap inHeap;
    int resident = 0;                         // admitted, not yet released
    std::vector<rr_ctx *> ctx;
    std::vector<cudaStream_t> stream;
    std::vector<Wave> wave;
    std::vector<rr_instance *> hDesc, dDesc;
    std::vector<uint8_t *> hStage;
    char *heapBase = nullptr;
    Heap heap;
    std::mutex mu;
    std::condition_variable cvWork, cvDone;
    std::deque<Req *> queued, planned;
    std::map<int64_t, Req *> reqs;
    int64_t nextTicket = 1;
    bool stop = false;
    int fatal = RR_OK;
    std::thread worker;
    Clock::time_point t0;
    double now() const { return std::chrono::duration<double, std::micro>(Clock::now() - t0).count(); }
};

static void finish(rr_server *S, Req *R, int status)
{
    if (status != RR_OK) R->desc.status = status;
    R->phase = DONE;
    R->tDone = S->now();
}

static void fail_all(rr_server *S, int status)
{
    S->fatal = status;
    for (auto &kv : S->reqs)
        if (kv.second->phase != DONE) finish(S, kv.second, status);
    S->queued.clear();
    S->planned.clear();
    S->cvDone.notify_all();
}

// One pass of the pipeline; returns true if it changed anything.
static bool pump(rr_server *S)
{
    bool did = false;
    const int NS = (int)S->stream.size();
    // 1. finished waves
    for (int s = 0; s < NS; ++s) {
        Wave &W = S->wave[s];
        if (!W.busy) continue;
        const cudaError_t q = cudaEventQuery(W.ev);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) { W.busy = false; fail_all(S, RR_ERR_CUDA); return true; }
        for (size_t i = 0; i < W.reqs.size(); ++i) {
            Req *R = W.reqs[i];
            R->desc = S->hDesc[s][i];
            if (W.kind == 1 && R->desc.status == RR_OK && (S->cfg.flags & RR_WITH_BATCH) && R->desc.n_moves > 0) {
                R->phase = PLANNED;
                S->planned.push_back(R);
            } else {
                finish(S, R, RR_OK);
            }
        }
        W.busy = false;
        W.reqs.clear();
        did = true;
        S->cvDone.notify_all();
    }
    if (S->stop) return did;
    // 2. batch waves for planned requests that fit in the heap (FIFO)
    for (int s = 0; s < NS && !S->planned.empty(); ++s) {
        Wave &W = S->wave[s];
        if (W.busy) continue;
        int cnt = 0;
        while (!S->planned.empty() && cnt < S->cfg.max_wave) {
            Req *R = S->planned.front();
            const int64_t steps = R->desc.n_steps;
            const int64_t bytes = 16 * std::max<int64_t>(steps, 1);
            if (Heap::round(bytes) > S->heap.size) {            // can never fit
                S->planned.pop_front();
                R->desc.n_ops = steps; R->desc.n_members = steps;
                finish(S, R, RR_ERR_CAPACITY);
                S->cvDone.notify_all();
                continue;
            }
            const int64_t off = S->heap.alloc(bytes);
            if (off < 0) break;                                  // wait for releases
            S->planned.pop_front();
            R->heapOff = off; R->heapBytes = bytes;
            rr_instance d = R->desc;
            d.ops = (rr_op *)(S->heapBase + off);
            d.cap_ops = steps;
            d.members = (int32_t *)(S->heapBase + off + 12 * steps);
            d.cap_members = steps;
            d.status = RR_OK;
            S->hDesc[s][cnt] = d;
            R->phase = BATCHING;
            W.reqs.push_back(R);
            ++cnt;
        }
        if (!cnt) continue;
        cudaStream_t st = S->stream[s];
        int e = cudaMemcpyAsync(S->dDesc[s], S->hDesc[s], sizeof(rr_instance) * cnt, cudaMemcpyHostToDevice, st);
        int r = e == cudaSuccess ? rr_plan_batched(S->ctx[s], S->dDesc[s], cnt, S->cfg.max_side, RR_BATCH_ONLY, st)
                                 : RR_ERR_CUDA;
        if (r == RR_OK) e = cudaMemcpyAsync(S->hDesc[s], S->dDesc[s], sizeof(rr_instance) * cnt, cudaMemcpyDeviceToHost, st);
        if (r == RR_OK && e == cudaSuccess) e = cudaEventRecord(W.ev, st);
        if (r != RR_OK || e != cudaSuccess) { fail_all(S, r != RR_OK ? r : RR_ERR_CUDA); return true; }
        W.busy = true; W.kind = 2;
        did = true;
    }
    // 3. plan waves for queued requests, admitted first come first served as
    // their grid and move list fit in the input pool
    for (int s = 0; s < NS && !S->queued.empty() && S->resident < S->cfg.slots; ++s) {
        Wave &W = S->wave[s];
        if (W.busy) continue;
        cudaStream_t st = S->stream[s];
        int cnt = 0, e = cudaSuccess;
        while (!S->queued.empty() && S->resident < S->cfg.slots && cnt < S->cfg.max_wave) {
            Req *R = S->queued.front();
            const int64_t gb = Heap::round((int64_t)R->grid.size());
            const int64_t cap = moves_cap(R->m, R->n);
            const int64_t bytes = gb + Heap::round(cap * (int64_t)sizeof(rr_move));
            const int64_t off = S->inHeap.alloc(bytes);
            if (off < 0) break;                                  // wait for releases
            S->queued.pop_front();
            R->inOff = off; R->inBytes = bytes;
            ++S->resident;
            R->tAdmit = S->now();
            uint8_t *stage = S->hStage[s] + (size_t)cnt * S->gridBytes;
            std::memcpy(stage, R->grid.data(), R->grid.size());
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(S->inBase + off, stage, R->grid.size(), cudaMemcpyHostToDevice, st);
            rr_instance d{};
            d.grid = S->inBase + off;
            d.layout = R->layout; d.m = R->m; d.n = R->n; d.rect = R->rect;
            d.moves = (rr_move *)(S->inBase + off + gb);
            d.cap_moves = cap;
            S->hDesc[s][cnt] = d;
            R->phase = PLANNING;
            W.reqs.push_back(R);
            ++cnt;
        }
        if (!cnt) break;                                         // the head of the queue does not fit yet
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(S->dDesc[s], S->hDesc[s], sizeof(rr_instance) * cnt, cudaMemcpyHostToDevice, st);
        int r = e == cudaSuccess ? rr_plan_batched(S->ctx[s], S->dDesc[s], cnt, S->cfg.max_side,
                                                        S->cfg.flags & (RR_BIRD | RR_STRICT_RESERVOIR), st) : RR_ERR_CUDA;
        if (r == RR_OK) e = cudaMemcpyAsync(S->hDesc[s], S->dDesc[s], sizeof(rr_instance) * cnt, cudaMemcpyDeviceToHost, st);
        if (r == RR_OK && e == cudaSuccess) e = cudaEventRecord(W.ev, st);
        if (r != RR_OK || e != cudaSuccess) { fail_all(S, r != RR_OK ? r : RR_ERR_CUDA); return true; }
        W.busy = true; W.kind = 1;
        did = true;
    }
    return did;
}

static void worker_main(rr_server *S)
{
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        const bool did = pump(S);
        bool busy = false;
        for (auto &W : S->wave) busy |= W.busy;
        if (S->stop && !busy) break;
        if (!did) {
            // waves in flight: poll their events at a short interval; idle: sleep until work arrives
            if (busy) S->cvWork.wait_for(lk, std::chrono::microseconds(20));
            else S->cvWork.wait_for(lk, std::chrono::milliseconds(2));
        }
    }
}

static void destroy(rr_server *S)
{
    for (auto *c : S->ctx) if (c) rr_ctx_destroy(c);
    for (auto s : S->stream) if (s) cudaStreamDestroy(s);
    for (auto &W : S->wave) if (W.ev) cudaEventDestroy(W.ev);
    for (auto *p : S->hDesc) if (p) cudaFreeHost(p);
    for (auto *p : S->dDesc) if (p) cudaFree(p);
    for (auto *p : S->hStage) if (p) cudaFreeHost(p);
    if (S->inBase) cudaFree(S->inBase);
    if (S->heapBase) cudaFree(S->heapBase);
    for (auto &kv : S->reqs) delete kv.second;
    delete S;
}

extern "C" int rr_serve_open(rr_server **out, const rr_serve_config *cfg)
{
    if (!out || !cfg || cfg->max_side < 1 || cfg->max_side > RR_MAX_SIDE || cfg->slots < 1 || cfg->streams < 1 ||
        cfg->streams > 64 || cfg->max_wave < 1 || cfg->max_wave > cfg->slots || cfg->max_wave > 65535 ||
        (cfg->flags & ~(RR_WITH_BATCH | RR_BIRD | RR_STRICT_RESERVOIR)) || cfg->heap_bytes < 0 || cfg->input_bytes < 0)
        return RR_ERR_ARG;
    *out = nullptr;
    rr_server *S = new (std::nothrow) rr_server();
    if (!S) return RR_ERR_ARG;
    S->cfg = *cfg;
    S->t0 = Clock::now();
    const int ms = cfg->max_side;
    S->gridBytes = std::max<int64_t>((int64_t)ms * ms, (int64_t)ms * ((ms + 31) / 32) * 4);
    bool ok = cudaGetDevice(&S->device) == cudaSuccess;
    // input pool: by default room for `slots` requests of the largest size
    const int64_t one = Heap::round(S->gridBytes) + Heap::round(moves_cap(ms, ms) * (int64_t)sizeof(rr_move));
    const int64_t pool = cfg->input_bytes > 0 ? cfg->input_bytes : one * cfg->slots;
    ok = ok && cudaMalloc(&S->inBase, pool) == cudaSuccess;
    S->inHeap.init(ok ? pool : 0);
    if (ok && cfg->heap_bytes > 0) ok = cudaMalloc(&S->heapBase, cfg->heap_bytes) == cudaSuccess;
    S->heap.init(ok ? cfg->heap_bytes : 0);
    S->ctx.assign(cfg->streams, nullptr);
    S->stream.assign(cfg->streams, nullptr);
    S->wave.resize(cfg->streams);
    S->hDesc.assign(cfg->streams, nullptr);
    S->dDesc.assign(cfg->streams, nullptr);
    S->hStage.assign(cfg->streams, nullptr);
    for (int s = 0; ok && s < cfg->streams; ++s) {
        ok = rr_ctx_create(&S->ctx[s], cfg->arena_bytes) == RR_OK && rr_internal_reserve(S->ctx[s], cfg->max_wave) == RR_OK &&
             cudaStreamCreateWithFlags(&S->stream[s], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&S->wave[s].ev, cudaEventDisableTiming) == cudaSuccess &&
             cudaMallocHost(&S->hDesc[s], sizeof(rr_instance) * cfg->max_wave) == cudaSuccess &&
             cudaMalloc(&S->dDesc[s], sizeof(rr_instance) * cfg->max_wave) == cudaSuccess &&
             cudaMallocHost(&S->hStage[s], (size_t)S->gridBytes * cfg->max_wave) == cudaSuccess;
    }
    if (!ok) { destroy(S); return RR_ERR_CUDA; }
    S->worker = std::thread(worker_main, S);
    *out = S;
    return RR_OK;
}

extern "C" int rr_serve_submit(rr_server *S, const void *h_grid, int layout, int m, int n, rr_rect rect,
                               int64_t *ticket)
{
    if (!S || !h_grid || !ticket || (layout != RR_U8 && layout != RR_BITS32) || m < 1 || n < 1 ||
        m > S->cfg.max_side || n > S->cfg.max_side || rect.r0 < 0 || rect.r0 >= rect.r1 || rect.r1 > m ||
        rect.c0 < 0 || rect.c0 >= rect.c1 || rect.c1 > n)
        return RR_ERR_ARG;
    Req *R = new (std::nothrow) Req();
    if (!R) return RR_ERR_ARG;
    const size_t bytes = layout == RR_U8 ? (size_t)m * n : (size_t)m * ((n + 31) / 32) * 4;
    if (Heap::round((int64_t)bytes) + Heap::round(moves_cap(m, n) * (int64_t)sizeof(rr_move)) > S->inHeap.size) {
        delete R;
        return RR_ERR_CAPACITY;                  // could never be admitted
    }
    R->grid.assign((const uint8_t *)h_grid, (const uint8_t *)h_grid + bytes);
    R->layout = layout; R->m = m; R->n = n; R->rect = rect;
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->fatal != RR_OK) { delete R; return S->fatal; }
    R->ticket = S->nextTicket++;
    R->tSubmit = S->now();
    R->desc.m = m; R->desc.n = n;
    S->reqs[R->ticket] = R;
    S->queued.push_back(R);
    *ticket = R->ticket;
    S->cvWork.notify_one();
    return RR_OK;
}

extern "C" int rr_serve_poll(rr_server *S, int64_t ticket, rr_serve_result *out, int64_t timeout_us)
{
    if (!S || !out) return RR_ERR_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return RR_ERR_ARG;
    Req *R = it->second;
    if (R->phase != DONE && timeout_us > 0)
        S->cvDone.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return R->phase == DONE; });
    if (R->phase != DONE) return RR_ERR_TIMEOUT;
    std::memset(out, 0, sizeof(*out));
    out->status = R->desc.status;
    out->m = R->m; out->n = R->n;
    out->n_moves = R->desc.n_moves; out->n_steps = R->desc.n_steps;
    out->n_ops = R->desc.n_ops; out->n_members = R->desc.n_members;
    out->d_moves = R->inOff >= 0 ? (const rr_move *)(S->inBase + R->inOff + Heap::round((int64_t)R->grid.size()))
                                 : nullptr;
    out->d_ops = R->heapOff >= 0 ? (const rr_op *)(S->heapBase + R->heapOff) : nullptr;
    out->d_members = R->heapOff >= 0 ? (const int32_t *)(S->heapBase + R->heapOff + 12 * R->desc.n_steps) : nullptr;
    out->t_submit_us = R->tSubmit; out->t_admit_us = R->tAdmit; out->t_done_us = R->tDone;
    return RR_OK;
}

extern "C" int rr_serve_release(rr_server *S, int64_t ticket)
{
    if (!S) return RR_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end() || it->second->phase != DONE) return RR_ERR_ARG;
    Req *R = it->second;
    if (R->inOff >= 0) { S->inHeap.release(R->inOff, R->inBytes); --S->resident; }
    if (R->heapOff >= 0) S->heap.release(R->heapOff, R->heapBytes);
    S->reqs.erase(it);
    delete R;
    S->cvWork.notify_one();
    return RR_OK;
}

extern "C" int rr_serve_close(rr_server *S)
{
    if (!S) return RR_ERR_ARG;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cvWork.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    destroy(S);
    return RR_OK;
}
