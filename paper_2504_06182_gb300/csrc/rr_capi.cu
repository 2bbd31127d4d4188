// rr_capi.cu -- the C ABI (include/rr.h): context, workspace arena and the
// launch sequences of the planner (Alg. 1) and the batching routine (Alg. 4).
#include <cstdio>
#include <cstring>
#include <cstdarg>
#include <algorithm>
#include <mutex>
#include "rr_internal.cuh"

namespace rrk {
__global__ void k_plan_setup(rr_instance *, JobWS *, int, int, Arena);
__global__ void k_transpose(rr_instance *, JobWS *, int);
__global__ void k_colstats(rr_instance *, JobWS *, int, int);
__global__ void k_pair(rr_instance *, JobWS *, int);
__global__ void k_emit_cols(rr_instance *, JobWS *, int);
__global__ void k_emit_recv(rr_instance *, JobWS *, int);
__global__ void k_bird(rr_instance *, JobWS *, int, int);
__global__ void k_bsetup(rr_instance *, JobWS *, int, Arena, int);
__global__ void k_pairoff_lookback(rr_instance *, JobWS *, int, Arena);
__global__ void k_gcount(rr_instance *, JobWS *, int);
__global__ void k_gscan(rr_instance *, JobWS *, int);
__global__ void k_gfill(rr_instance *, JobWS *, int);
__global__ void k_gsort(rr_instance *, JobWS *, int, int);
__global__ void k_gsweep_h(rr_instance *, JobWS *, int, int);
__global__ void k_gsweep_v(rr_instance *, JobWS *, int, int);
__global__ void k_bsucc(rr_instance *, JobWS *, int);
__global__ void k_brec(rr_instance *, JobWS *, int);
__global__ void k_classify(rr_instance *, int, int, int, int *, int *);
__global__ void k_order(const rr_instance *, int, int *);
__global__ void k_gather(const rr_instance *, const int *, rr_instance *);
__global__ void k_scatter(rr_instance *, const int *, const rr_instance *, int);
__global__ void k_sim16(rr_instance *, JobWS *, int, const int *, const int *, int, int);
__global__ void k_sim32(rr_instance *, JobWS *, int, const int *, const int *, int, int);
__global__ void k_sim16w(rr_instance *, JobWS *, int, const int *, const int *, int, int);
__global__ void k_sim32w(rr_instance *, JobWS *, int, const int *, const int *, int, int);
}  // namespace rrk

using namespace rrk;

static_assert(sizeof(rr_instance) == 128, "rr_instance layout is part of the ABI");

// Calls over at most this many grids run the simulation as one size class.
static constexpr int SMALL_CALL = 8;

// Kernels launched with more than the default 48 KB of dynamic shared memory.
enum { SM_GSORT, SM_GSWEEP_H, SM_GSWEEP_V, SM_SIM16, SM_SIM32, SM_SIM16W, SM_SIM32W, SM_BIRD, SM_ONE, SM_NKERNEL };

struct rr_ctx {
    int device;
    int nsm;                     // streaming multiprocessors of the device
    int smemLimit[SM_NKERNEL];   // dynamic shared memory each of those kernels may request
    char *arena;
    unsigned long long arena_size;
    unsigned long long *d_top;
    rr_instance *d_one;       // descriptor slot of the single-grid entry points
    rr_instance *h_one;       // rr_plan_one: the final descriptor, written by the kernel (mapped host memory)
    rr_instance *d_hone;      // its device address
    JobWS *d_ws;
    int ws_cap;
    char err[256];
    // simulation size classes: side bounds, counts and lists (device), and a
    // stream per class forked from / joined into the caller's stream
    static const int MAXCLASS = 8;
    // launch configuration of batched calls (rr_autotune may change it):
    // simulation size classes, and per-grid block budgets scaled by 2^shift
    int nclass = 4, shift = 0;
    int pipe;                    // batched calls: pipeline split (index into PIPE_SPLITS; 0: none)
    // pipeline by size: sorted descriptor copy; a stream per leading group
    // (priorities descending) and one for the rest
    static const int MAXLEAD = 4;
    rr_instance *d_pinst;
    int *d_perm;
    cudaStream_t leadStream[MAXLEAD], restStream;
    cudaEvent_t evStart, evLead[MAXLEAD], evRest, evSim[MAXLEAD];
    int quiet;                   // no stage marks (the second pipeline)
    int *d_classCount, *d_classList;
    int classListCap;
    cudaStream_t classStream[MAXCLASS];
    cudaEvent_t evFork, evJoin[MAXCLASS];
    int64_t nlaunch;             // kernels launched so far
    // RR_GRAPH: the captured launch sequence and the call it belongs to
    cudaStream_t capStream;
    cudaGraphExec_t graph;
    rr_instance *gInst;
    int gCount, gMaxSide, gFlags;
    int64_t gLaunches;
    int capturing;
    // stage tracing: events recorded on the launching stream around every kernel
    int tracing;
    int nmarks;
    cudaEvent_t marks[32];
    const char *names[32];
};

static void mark(rr_ctx *ctx, cudaStream_t s, const char *name)
{
    if (!ctx->tracing || ctx->capturing || ctx->quiet || ctx->nmarks >= 32) return;
    if (!ctx->marks[ctx->nmarks]) cudaEventCreate(&ctx->marks[ctx->nmarks]);
    cudaEventRecord(ctx->marks[ctx->nmarks], s);
    ctx->names[ctx->nmarks] = name;
    ++ctx->nmarks;
}

// error text of calls without a context (per thread: calls may come from several)
static thread_local char g_err[256] = "";

static int fail(rr_ctx *ctx, int code, const char *fmt, ...)
{
    char *dst = ctx ? ctx->err : g_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 256, fmt, ap);
    va_end(ap);
    return code;
}

#define CUDA_TRY(call)                                                                    \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) return fail(ctx, RR_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// Dynamic shared-memory limits are function attributes shared by every host
// thread and every context of the process. They are set once per device, to
// the device's opt-in maximum, before the first launch, and never changed:
// setting them per launch would race with launches of the same kernels from
// other threads (a server's worker next to a caller's own context), and a
// lowered limit would break a launch that another thread already sized.
static std::mutex g_limits_mu;
static constexpr int MAX_DEVICES = 64;
static bool g_limits_set[MAX_DEVICES];
static int g_limits[MAX_DEVICES][SM_NKERNEL];

static int smem_limits(int dev, int *out)
{
    if (dev < 0 || dev >= MAX_DEVICES) return fail(nullptr, RR_ERR_CUDA, "device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_limits_mu);
    if (!g_limits_set[dev]) {
        int optin = 0;
        cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        const void *fn[SM_NKERNEL] = {(const void *)k_gsort, (const void *)k_gsweep_h, (const void *)k_gsweep_v,
                                      (const void *)k_sim16, (const void *)k_sim32, (const void *)k_sim16w,
                                      (const void *)k_sim32w, (const void *)k_bird, one_kernel()};
        for (int i = 0; e == cudaSuccess && i < SM_NKERNEL; ++i) {
            cudaFuncAttributes fa;
            e = cudaFuncGetAttributes(&fa, fn[i]);
            if (e != cudaSuccess) break;
            const int lim = optin - (int)fa.sharedSizeBytes;
            e = cudaFuncSetAttribute(fn[i], cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
            g_limits[dev][i] = lim;
        }
        if (e != cudaSuccess) return fail(nullptr, RR_ERR_CUDA, "shared-memory limits: %s", cudaGetErrorString(e));
        g_limits_set[dev] = true;
    }
    std::memcpy(out, g_limits[dev], sizeof(g_limits[dev]));
    return RR_OK;
}

static void drop_graph(rr_ctx *ctx)
{
    if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
    ctx->graph = nullptr;
    ctx->gInst = nullptr;
}

static int ensure_ws(rr_ctx *ctx, int count)
{
    if (count <= ctx->ws_cap) return RR_OK;
    drop_graph(ctx);          // it refers to the old table
    int cap = std::max(count, 2 * ctx->ws_cap);
    if (ctx->d_ws) CUDA_TRY(cudaFree(ctx->d_ws));
    ctx->d_ws = nullptr;
    ctx->ws_cap = 0;
    CUDA_TRY(cudaMalloc(&ctx->d_ws, sizeof(JobWS) * (size_t)cap));
    if (ctx->d_classList) CUDA_TRY(cudaFree(ctx->d_classList));
    ctx->d_classList = nullptr;
    CUDA_TRY(cudaMalloc(&ctx->d_classList, sizeof(int) * (size_t)cap * rr_ctx::MAXCLASS));
    if (ctx->d_pinst) CUDA_TRY(cudaFree(ctx->d_pinst));
    if (ctx->d_perm) CUDA_TRY(cudaFree(ctx->d_perm));
    ctx->d_pinst = nullptr;
    ctx->d_perm = nullptr;
    CUDA_TRY(cudaMalloc(&ctx->d_pinst, sizeof(rr_instance) * (size_t)cap));
    CUDA_TRY(cudaMalloc(&ctx->d_perm, sizeof(int) * (size_t)cap));
    ctx->ws_cap = cap;
    return RR_OK;
}

extern "C" int rr_ctx_create(rr_ctx **out, int64_t arena_bytes)
{
    rr_ctx *ctx = nullptr;
    if (!out) return fail(nullptr, RR_ERR_ARG, "rr_ctx_create: null output pointer");
    *out = nullptr;
    ctx = new (std::nothrow) rr_ctx();   // value-initialised: every member zero, then its initialiser
    if (!ctx) return fail(nullptr, RR_ERR_ARG, "rr_ctx_create: out of host memory");
    ctx->nclass = 4;
    ctx->shift = 0;
    ctx->pipe = 1;
    if (arena_bytes <= 0) arena_bytes = 1ll << 30;
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->arena, (size_t)arena_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_top, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_one, sizeof(rr_instance));
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&ctx->h_one, sizeof(rr_instance), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&ctx->d_hone, ctx->h_one, 0);
    if (e != cudaSuccess) {
        fail(nullptr, RR_ERR_CUDA, "rr_ctx_create: %s", cudaGetErrorString(e));
        if (ctx->arena) cudaFree(ctx->arena);
        if (ctx->d_top) cudaFree(ctx->d_top);
        if (ctx->d_one) cudaFree(ctx->d_one);
        if (ctx->h_one) cudaFreeHost(ctx->h_one);
        delete ctx;
        return RR_ERR_CUDA;
    }
    ctx->arena_size = (unsigned long long)arena_bytes;
    int st = smem_limits(ctx->device, ctx->smemLimit);
    if (st != RR_OK) { rr_ctx_destroy(ctx); return st; }
    st = ensure_ws(ctx, 1);
    if (st != RR_OK) { rr_ctx_destroy(ctx); return st; }
    bool ok = cudaMalloc(&ctx->d_classCount, sizeof(int) * rr_ctx::MAXCLASS) == cudaSuccess &&
              cudaEventCreateWithFlags(&ctx->evFork, cudaEventDisableTiming) == cudaSuccess &&
              cudaStreamCreateWithFlags(&ctx->capStream, cudaStreamNonBlocking) == cudaSuccess;
    // class streams get priorities by class, the largest grids highest: their
    // simulations are the longest, so their blocks should start first (this
    // also holds inside a captured graph, instantiated with node priorities)
    int least = 0, greatest = 0;
    ok = ok && cudaDeviceGetStreamPriorityRange(&least, &greatest) == cudaSuccess;
    ok = ok && cudaStreamCreateWithPriority(&ctx->restStream, cudaStreamNonBlocking, least) == cudaSuccess &&
         cudaEventCreateWithFlags(&ctx->evStart, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&ctx->evRest, cudaEventDisableTiming) == cudaSuccess;
    for (int g = 0; ok && g < rr_ctx::MAXLEAD; ++g) {
        const int prio = greatest + (least - greatest) * g / rr_ctx::MAXLEAD;
        ok = cudaStreamCreateWithPriority(&ctx->leadStream[g], cudaStreamNonBlocking, prio) == cudaSuccess &&
             cudaEventCreateWithFlags(&ctx->evLead[g], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&ctx->evSim[g], cudaEventDisableTiming) == cudaSuccess;
    }
    for (int c = 0; ok && c < rr_ctx::MAXCLASS; ++c) {
        const int prio = least + (greatest - least) * c / (rr_ctx::MAXCLASS - 1);
        ok = cudaStreamCreateWithPriority(&ctx->classStream[c], cudaStreamNonBlocking, prio) == cudaSuccess &&
             cudaEventCreateWithFlags(&ctx->evJoin[c], cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) { rr_ctx_destroy(ctx); return fail(nullptr, RR_ERR_CUDA, "rr_ctx_create: stream/event setup failed"); }
    *out = ctx;
    return RR_OK;
}

extern "C" int rr_ctx_destroy(rr_ctx *ctx)
{
    if (!ctx) return RR_ERR_ARG;
    cudaFree(ctx->arena);
    cudaFree(ctx->d_top);
    cudaFree(ctx->d_one);
    if (ctx->h_one) cudaFreeHost(ctx->h_one);
    cudaFree(ctx->d_ws);
    drop_graph(ctx);
    if (ctx->capStream) cudaStreamDestroy(ctx->capStream);
    if (ctx->restStream) cudaStreamDestroy(ctx->restStream);
    for (cudaEvent_t e : {ctx->evStart, ctx->evRest}) if (e) cudaEventDestroy(e);
    for (int g = 0; g < rr_ctx::MAXLEAD; ++g) {
        if (ctx->leadStream[g]) cudaStreamDestroy(ctx->leadStream[g]);
        if (ctx->evLead[g]) cudaEventDestroy(ctx->evLead[g]);
        if (ctx->evSim[g]) cudaEventDestroy(ctx->evSim[g]);
    }
    cudaFree(ctx->d_pinst);
    cudaFree(ctx->d_perm);
    cudaFree(ctx->d_classCount);
    cudaFree(ctx->d_classList);
    if (ctx->evFork) cudaEventDestroy(ctx->evFork);
    for (int c = 0; c < rr_ctx::MAXCLASS; ++c) {
        if (ctx->classStream[c]) cudaStreamDestroy(ctx->classStream[c]);
        if (ctx->evJoin[c]) cudaEventDestroy(ctx->evJoin[c]);
    }
    for (int i = 0; i < 32; ++i) if (ctx->marks[i]) cudaEventDestroy(ctx->marks[i]);
    delete ctx;
    return RR_OK;
}

extern "C" int rr_launch_count(rr_ctx *ctx, int64_t *launches)
{
    if (!ctx || !launches) return RR_ERR_ARG;
    *launches = ctx->nlaunch;
    return RR_OK;
}

extern "C" const char *rr_last_error(rr_ctx *ctx) { return ctx ? ctx->err : g_err; }

static Arena arena_of(rr_ctx *ctx)
{
    Arena A;
    A.base = ctx->arena;
    A.size = ctx->arena_size;
    A.top = ctx->d_top;
    return A;
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Blocks a launch may spread over all grids of a call (divided by the count).
static int budget(const rr_ctx *ctx, int base) { return ctx->shift >= 0 ? base << ctx->shift : base >> -ctx->shift; }

// Shared memory of a k_bird block: reservoir-row bits of the largest grid
// (column-major, one word per 32 rows), the two token lists (each the next
// power of two >= max_side: they double as sort buffers), then five int16
// arrays of max_side (the receiver list: columns, band atoms, atoms above
// the band; the current receiver's band holes and band atom rows).
static size_t bird_smem_bytes(int max_side)
{
    size_t cap = 1;
    while (cap < (size_t)max_side) cap <<= 1;
    return 4 * ((size_t)max_side * ((max_side + 31) / 32) + 2 * cap) + 2 * 5 * (size_t)max_side;
}

// Planning kernels over `count` device descriptors whose sides are <= max_side:
// red-rec (Alg. 1), or with RR_BIRD the bird algorithm (Alg. 2), which shares
// red-rec's column phase; RR_STRICT_RESERVOIR selects the strict reading of
// target sub-rectangles for either.
static int launch_plan(rr_ctx *ctx, rr_instance *d_inst, JobWS *ws, int count, int max_side, cudaStream_t s,
                       int flags)
{
    const bool bird = (flags & RR_BIRD) != 0;
    const int strict = (flags & RR_STRICT_RESERVOIR) ? 1 : 0;
    const Arena A = arena_of(ctx);
    const int colBlocks = clampi(std::max(1, budget(ctx, 4096) / count), 1, (max_side + 7) / 8);
    const int tiles = ((max_side + 31) / 32) * ((max_side + 31) / 32);
    const int trBlocks = clampi(std::max(1, budget(ctx, 4096) / count), 1, (tiles + 7) / 8);
    const int recvBlocks = clampi(std::max(1, budget(ctx, 2048) / count), 1, max_side);
    mark(ctx, s, "k_plan_setup");
    k_plan_setup<<<(count + 127) / 128, 128, 0, s>>>(d_inst, ws, count, max_side, A);
    mark(ctx, s, "k_transpose");
    k_transpose<<<dim3(trBlocks, count), 256, 0, s>>>(d_inst, ws, count);
    mark(ctx, s, "k_colstats");
    k_colstats<<<dim3(colBlocks, count), 256, 0, s>>>(d_inst, ws, count, strict);
    if (bird) {
        const size_t birdSmem = bird_smem_bytes(max_side);
        if (birdSmem > (size_t)ctx->smemLimit[SM_BIRD])
            return fail(ctx, RR_ERR_ARG, "bird: shared memory %zu for side %d too large", birdSmem, max_side);
        mark(ctx, s, "k_bird");
        k_bird<<<count, 64, birdSmem, s>>>(d_inst, ws, count, max_side);
        mark(ctx, s, "k_emit_cols");
        k_emit_cols<<<dim3(colBlocks, count), 256, 0, s>>>(d_inst, ws, count);
        mark(ctx, s, nullptr);
        CUDA_TRY(cudaGetLastError());
        ctx->nlaunch += 5;
        return RR_OK;
    }
    const size_t pairSmem = (size_t)max_side * 30 + 64;
    mark(ctx, s, "k_pair");
    k_pair<<<count, 32, pairSmem, s>>>(d_inst, ws, count);
    mark(ctx, s, "k_emit_cols");
    k_emit_cols<<<dim3(colBlocks, count), 256, 0, s>>>(d_inst, ws, count);
    mark(ctx, s, "k_emit_recv");
    k_emit_recv<<<dim3(recvBlocks, count), 256, 0, s>>>(d_inst, ws, count);
    mark(ctx, s, nullptr);
    CUDA_TRY(cudaGetLastError());
    ctx->nlaunch += 6;
    return RR_OK;
}

// Simulation launch shapes: per size class on forked streams, or one launch
// over every instance of the call on its stream.
enum { SIM_CLASSES = 0, SIM_ONE = 1 };

// Batching kernels. Before the simulation the stream waits for `waitSim`
// and records `atSim` (either may be null).
static int launch_batch(rr_ctx *ctx, rr_instance *d_inst, JobWS *ws, int count, int max_side, cudaStream_t s,
                        int simMode, cudaEvent_t waitSim, cudaEvent_t atSim)
{
    const Arena A = arena_of(ctx);
    const int pathBlocks = clampi(std::max(1, budget(ctx, 8192) / count), 1, 512);
    // move lists long enough for it (grids above 256 on a side) get their
    // path-vertex offsets from the multi-block look-back scan
    const int lookback = max_side > 256 ? 1 : 0;
    mark(ctx, s, "k_bsetup");
    k_bsetup<<<count, 512, 0, s>>>(d_inst, ws, count, A, lookback);
    if (lookback) {
        mark(ctx, s, "k_pairoff_lookback");
        k_pairoff_lookback<<<dim3(clampi(2 * ctx->nsm / count, 1, 2 * ctx->nsm), count), LB_THREADS, 0, s>>>(
            d_inst, ws, count, A);
        ctx->nlaunch += 1;
    }
    {
        // Gamma by column and row sweeps
        const int lineBlocks = clampi(std::max(1, budget(ctx, 8192) / count), 1, (2 * max_side + 7) / 8);
        mark(ctx, s, "k_gcount");
        k_gcount<<<dim3(pathBlocks, count), 256, 0, s>>>(d_inst, ws, count);
        mark(ctx, s, "k_gscan");
        k_gscan<<<count, 64, 0, s>>>(d_inst, ws, count);
        mark(ctx, s, "k_gfill");
        k_gfill<<<dim3(pathBlocks, count), 256, 0, s>>>(d_inst, ws, count);
        int P2 = 32;
        while (P2 < max_side) P2 <<= 1;
        if (8 * 4 * P2 > ctx->smemLimit[SM_GSORT] || 8 * 4 * max_side > ctx->smemLimit[SM_GSWEEP_H] ||
            8 * 12 * max_side > ctx->smemLimit[SM_GSWEEP_V])
            return fail(ctx, RR_ERR_ARG, "Gamma sweeps: shared memory for side %d too large", max_side);
        mark(ctx, s, "k_gsort");
        k_gsort<<<dim3(lineBlocks, count), 256, 8 * 4 * (size_t)P2, s>>>(d_inst, ws, count, P2);
        mark(ctx, s, "k_gsweep_h");
        k_gsweep_h<<<dim3(lineBlocks, count), 256, 8 * 4 * (size_t)max_side, s>>>(d_inst, ws, count, max_side);
        mark(ctx, s, "k_gsweep_v");
        k_gsweep_v<<<dim3(lineBlocks, count), 256, 8 * 12 * (size_t)max_side, s>>>(d_inst, ws, count, max_side);
    }
    mark(ctx, s, "k_bsucc");
    k_bsucc<<<dim3(pathBlocks, count), 256, 0, s>>>(d_inst, ws, count);
    mark(ctx, s, "k_brec");
    k_brec<<<dim3(pathBlocks, count), 256, 0, s>>>(d_inst, ws, count);
    // simulation: one warp per instance, launched per size class on forked
    // streams so that each class's shared memory fits its own grids; slot
    // table, static lists and buffers live in shared memory (layout mirrored
    // in k_sim)
    // one launch over all instances (a small call, or the largest grids of a
    // pipelined call), or size classes each on a stream of its own so that
    // each gets shared memory for its own sides
    const bool one = simMode == SIM_ONE || count <= SMALL_CALL;
    const int nclass = one ? 1 : ctx->nclass;
    if (!one) {
        CUDA_TRY(cudaMemsetAsync(ctx->d_classCount, 0, sizeof(int) * rr_ctx::MAXCLASS, s));
        mark(ctx, s, "k_classify");
        k_classify<<<(count + 255) / 256, 256, 0, s>>>(d_inst, count, nclass, max_side, ctx->d_classCount,
                                                      ctx->d_classList);
    }
    if (waitSim) CUDA_TRY(cudaStreamWaitEvent(s, waitSim, 0));
    if (atSim) CUDA_TRY(cudaEventRecord(atSim, s));
    mark(ctx, s, "k_sim");
    if (!one) CUDA_TRY(cudaEventRecord(ctx->evFork, s));
    for (int c = nclass - 1; c >= 0; --c) {
        cudaStream_t cs = one ? s : ctx->classStream[c];
        if (!one) CUDA_TRY(cudaStreamWaitEvent(cs, ctx->evFork, 0));
        const int side = class_side(max_side, c, nclass);
        // ready moves never exceed two per column here (one chain head each
        // way); beyond the capacity slots spill to the global overflow area
        const int slotCap = 2 * side + 8, lineCap = side;
        // links are 16-bit up to side 256: about 2 * side moves are ready at
        // once, far below 32 768; an instance that would need more slots
        // ends with an internal error instead of wrapping an index
        const bool narrow = lineCap <= 256;
        const size_t simSmem = sim_smem_bytes(slotCap, lineCap, narrow ? 2 : 4);
        if (simSmem > (size_t)std::min(ctx->smemLimit[narrow ? SM_SIM16 : SM_SIM32],
                                       ctx->smemLimit[narrow ? SM_SIM16W : SM_SIM32W]))
            return fail(ctx, RR_ERR_ARG, "simulation shared memory %zu too large", simSmem);
        const int *list = one ? nullptr : ctx->d_classList + (size_t)c * count;
        const int *cnt = one ? nullptr : ctx->d_classCount + c;
        // the narrow pass, then the wide one for the instances it handed over
        // (its blocks of other instances return at once)
        if (narrow) {
            k_sim16<<<count, 32, simSmem, cs>>>(d_inst, ws, count, list, cnt, slotCap, lineCap);
            k_sim16w<<<count, 32, simSmem, cs>>>(d_inst, ws, count, list, cnt, slotCap, lineCap);
        } else {
            k_sim32<<<count, 32, simSmem, cs>>>(d_inst, ws, count, list, cnt, slotCap, lineCap);
            k_sim32w<<<count, 32, simSmem, cs>>>(d_inst, ws, count, list, cnt, slotCap, lineCap);
        }
        if (!one) {
            CUDA_TRY(cudaEventRecord(ctx->evJoin[c], cs));
            CUDA_TRY(cudaStreamWaitEvent(s, ctx->evJoin[c], 0));
        }
    }
    mark(ctx, s, nullptr);
    CUDA_TRY(cudaGetLastError());
    ctx->nlaunch += (one ? 9 : 10) + 2 * nclass;
    return RR_OK;
}

static bool rect_ok(int m, int n, rr_rect R)
{
    return m >= 1 && n >= 1 && m <= RR_MAX_SIDE && n <= RR_MAX_SIDE && R.r0 >= 0 && R.r0 < R.r1 &&
           R.r1 <= m && R.c0 >= 0 && R.c0 < R.c1 && R.c1 <= n;
}

static int plan_one(rr_ctx *ctx, const void *d_grid, int layout, int m, int n, rr_rect rect, rr_move *d_moves,
                    int64_t cap, int64_t *n_moves, cudaStream_t stream, int flags, const char *name)
{
    if (!ctx || !d_grid || !n_moves || (layout != RR_U8 && layout != RR_BITS32) || !rect_ok(m, n, rect) ||
        cap < 0 || (cap > 0 && !d_moves) || (flags & ~(RR_BIRD | RR_STRICT_RESERVOIR)))
        return fail(ctx, RR_ERR_ARG, "%s: bad argument (m=%d n=%d rect=[%d,%d,%d,%d] layout=%d cap=%lld flags=%d)",
                    name, m, n, rect.r0, rect.c0, rect.r1, rect.c1, layout, (long long)cap, flags);
    rr_instance h;
    std::memset(&h, 0, sizeof(h));
    h.grid = d_grid; h.layout = layout; h.m = m; h.n = n; h.rect = rect;
    h.moves = d_moves; h.cap_moves = cap;
    ctx->nmarks = 0;
    CUDA_TRY(cudaMemsetAsync(ctx->d_top, 0, sizeof(unsigned long long), stream));
    CUDA_TRY(cudaMemcpyAsync(ctx->d_one, &h, sizeof(h), cudaMemcpyHostToDevice, stream));
    int st = launch_plan(ctx, ctx->d_one, ctx->d_ws, 1, std::max(m, n), stream, flags);
    if (st != RR_OK) return st;
    CUDA_TRY(cudaMemcpyAsync(&h, ctx->d_one, sizeof(h), cudaMemcpyDeviceToHost, stream));
    CUDA_TRY(cudaStreamSynchronize(stream));
    *n_moves = h.n_moves;
    if (h.status < 0)
        return fail(ctx, h.status, "%s: device status %d (n_moves=%lld)", name, h.status, (long long)h.n_moves);
    return h.status;
}

extern "C" int rr_plan(rr_ctx *ctx, const void *d_grid, int layout, int m, int n, rr_rect rect,
                       rr_move *d_moves, int64_t cap, int64_t *n_moves, cudaStream_t stream)
{
    return plan_one(ctx, d_grid, layout, m, n, rect, d_moves, cap, n_moves, stream, 0, "rr_plan");
}

extern "C" int rr_bird_plan(rr_ctx *ctx, const void *d_grid, int layout, int m, int n, rr_rect rect,
                            rr_move *d_moves, int64_t cap, int64_t *n_moves, cudaStream_t stream)
{
    return plan_one(ctx, d_grid, layout, m, n, rect, d_moves, cap, n_moves, stream, RR_BIRD, "rr_bird_plan");
}

extern "C" int rr_plan_mode(rr_ctx *ctx, const void *d_grid, int layout, int m, int n, rr_rect rect, int flags,
                            rr_move *d_moves, int64_t cap, int64_t *n_moves, cudaStream_t stream)
{
    return plan_one(ctx, d_grid, layout, m, n, rect, d_moves, cap, n_moves, stream, flags, "rr_plan_mode");
}

extern "C" int rr_batch(rr_ctx *ctx, const rr_move *d_moves, int64_t n_moves, int m, int n, rr_op *d_ops,
                        int64_t cap_ops, int32_t *d_members, int64_t cap_members, int64_t *n_ops,
                        int64_t *n_members, cudaStream_t stream)
{
    if (!ctx || !n_ops || !n_members || m < 1 || n < 1 || m > RR_MAX_SIDE || n > RR_MAX_SIDE || n_moves < 0 ||
        n_moves > 0x3fffffff || (n_moves > 0 && !d_moves) || cap_ops < 0 || cap_members < 0)
        return fail(ctx, RR_ERR_ARG, "rr_batch: bad argument (m=%d n=%d n_moves=%lld)", m, n, (long long)n_moves);
    rr_instance h;
    std::memset(&h, 0, sizeof(h));
    h.grid = d_moves; h.layout = RR_U8; h.m = m; h.n = n;
    h.rect = rr_rect{0, 0, m, n};
    h.moves = const_cast<rr_move *>(d_moves); h.n_moves = n_moves; h.cap_moves = n_moves;
    h.ops = d_ops; h.cap_ops = cap_ops; h.members = d_members; h.cap_members = cap_members;
    h.status = RR_OK;
    ctx->nmarks = 0;
    CUDA_TRY(cudaMemsetAsync(ctx->d_top, 0, sizeof(unsigned long long), stream));
    CUDA_TRY(cudaMemcpyAsync(ctx->d_one, &h, sizeof(h), cudaMemcpyHostToDevice, stream));
    int st = launch_batch(ctx, ctx->d_one, ctx->d_ws, 1, std::max(m, n), stream, SIM_ONE, nullptr, nullptr);
    if (st != RR_OK) return st;
    CUDA_TRY(cudaMemcpyAsync(&h, ctx->d_one, sizeof(h), cudaMemcpyDeviceToHost, stream));
    CUDA_TRY(cudaStreamSynchronize(stream));
    *n_ops = h.n_ops;
    *n_members = h.n_members;
    if (h.status < 0) return fail(ctx, h.status, "rr_batch: device status %d", h.status);
    return h.status;
}

extern "C" int rr_plan_one(rr_ctx *ctx, const void *d_grid, int layout, int m, int n, rr_rect rect, int flags,
                           rr_move *d_moves, int64_t cap_moves, rr_op *d_ops, int64_t cap_ops, int32_t *d_members,
                           int64_t cap_members, int64_t *counts, cudaStream_t stream)
{
    const bool batch = (flags & RR_WITH_BATCH) != 0;
    if (!ctx || !d_grid || !counts || (layout != RR_U8 && layout != RR_BITS32) || !rect_ok(m, n, rect) ||
        m > ONE_MAX_SIDE || n > ONE_MAX_SIDE || cap_moves < 0 || (cap_moves > 0 && !d_moves) ||
        (flags & ~(RR_WITH_BATCH | RR_BIRD | RR_STRICT_RESERVOIR)) ||
        (batch && (cap_ops < 0 || cap_members < 0 || (cap_ops > 0 && !d_ops) || (cap_members > 0 && !d_members))))
        return fail(ctx, RR_ERR_ARG, "rr_plan_one: bad argument (m=%d n=%d rect=[%d,%d,%d,%d] layout=%d flags=%d)",
                    m, n, rect.r0, rect.c0, rect.r1, rect.c1, layout, flags);
    const int side = std::max(m, n);
    const size_t smem = one_smem_bytes(side, flags);
    if (smem > (size_t)ctx->smemLimit[SM_ONE])
        return fail(ctx, RR_ERR_ARG, "rr_plan_one: shared memory %zu for side %d too large", smem, side);
    rr_instance h;
    std::memset(&h, 0, sizeof(h));
    h.grid = d_grid; h.layout = layout; h.m = m; h.n = n; h.rect = rect;
    h.moves = d_moves; h.cap_moves = cap_moves;
    if (batch) { h.ops = d_ops; h.cap_ops = cap_ops; h.members = d_members; h.cap_members = cap_members; }
    ctx->nmarks = 0;
    mark(ctx, stream, "k_one");
    if (one_launch(h, ctx->d_one, ctx->d_ws, arena_of(ctx), flags, side, smem, ctx->d_hone, stream) != RR_OK)
        return fail(ctx, RR_ERR_CUDA, "rr_plan_one: launch: %s", cudaGetErrorString(cudaGetLastError()));
    mark(ctx, stream, nullptr);
    ctx->nlaunch += 1;
    CUDA_TRY(cudaStreamSynchronize(stream));
    const volatile rr_instance *r = ctx->h_one;
    counts[0] = r->n_moves;
    counts[1] = r->n_steps;
    counts[2] = batch ? r->n_ops : 0;
    counts[3] = batch ? r->n_members : 0;
    const int st = r->status;
    if (st < 0 && st != RR_ERR_CAPACITY)
        return fail(ctx, st, "rr_plan_one: device status %d (n_moves=%lld)", st, (long long)counts[0]);
    return st;
}

// Calls over at least this many grids, with batching, may run pipelined.
static constexpr int PIPE_MIN = 256;
// Pipeline splits: the leading groups end at these fractions of the grids
// (ordered by side, largest first); the rest forms the last group.
// (in 64ths of the call's grids)
static constexpr int PIPE_SPLITS = 5;
static const int PIPE_FRAC64[PIPE_SPLITS][rr_ctx::MAXLEAD] = {
    {0, 0, 0, 0},          // none
    {16, 0, 0, 0},         // the largest quarter, then the rest
    {4, 16, 0, 0},         // 1/16, 1/4
    {4, 8, 16, 32},        // 1/16, 1/8, 1/4, 1/2
    {1, 4, 16, 0},         // 1/64, 1/16, 1/4
};

// The whole sequence of one rr_plan_batched call on `stream`.
//
// With batching, a call over many grids can run pipelined by size: the
// grids are ordered by side, largest first, into a descriptor copy; each
// leading group is planned, given its conflict graph and simulated (one
// launch) on a stream of its own, priorities descending, and the rest goes
// through planning and graph construction meanwhile on a low-priority stream
// and is simulated by size class. A group's simulations start once the
// previous group's have started, so the largest grids, whose simulations
// are the longest, start first instead of after every grid's graph.
static int launch_sequence(rr_ctx *ctx, rr_instance *d_inst, int count, int max_side, int flags,
                           cudaStream_t stream)
{
    CUDA_TRY(cudaMemsetAsync(ctx->d_top, 0, sizeof(unsigned long long), stream));
    const bool plan = !(flags & RR_BATCH_ONLY), batch = (flags & (RR_WITH_BATCH | RR_BATCH_ONLY)) != 0;
    const int pflags = flags & (RR_BIRD | RR_STRICT_RESERVOIR);
    const int *frac = PIPE_FRAC64[ctx->pipe > 0 && ctx->pipe < PIPE_SPLITS ? ctx->pipe : 0];
    if (!batch || frac[0] == 0 || count < PIPE_MIN) {
        int st = plan ? launch_plan(ctx, d_inst, ctx->d_ws, count, max_side, stream, pflags) : RR_OK;
        if (st == RR_OK && batch)
            st = launch_batch(ctx, d_inst, ctx->d_ws, count, max_side, stream, SIM_CLASSES, nullptr, nullptr);
        return st;
    }
    mark(ctx, stream, "k_order");
    k_order<<<1, 1024, 0, stream>>>(d_inst, count, ctx->d_perm);
    mark(ctx, stream, "k_gather");
    k_gather<<<count, 32, 0, stream>>>(d_inst, ctx->d_perm, ctx->d_pinst);
    CUDA_TRY(cudaEventRecord(ctx->evStart, stream));
    int st = RR_OK, lo = 0, ng = 0;
    cudaEvent_t prevSim = nullptr;
    for (int g = 0; g < rr_ctx::MAXLEAD && frac[g] && st == RR_OK; ++g) {
        const int hi = std::max(lo + 1, (int)((int64_t)count * frac[g] / 64));
        if (hi >= count) break;
        cudaStream_t gs = ctx->leadStream[g];
        CUDA_TRY(cudaStreamWaitEvent(gs, ctx->evStart, 0));
        ctx->quiet = g > 0;                  // stage marks follow the first group
        if (plan) st = launch_plan(ctx, ctx->d_pinst + lo, ctx->d_ws + lo, hi - lo, max_side, gs, pflags);
        if (st == RR_OK)
            st = launch_batch(ctx, ctx->d_pinst + lo, ctx->d_ws + lo, hi - lo, max_side, gs, SIM_ONE, prevSim,
                              ctx->evSim[g]);
        // the "k_sim" stage runs on to the join after every simulation (drop
        // the first group's end-of-sequence mark)
        if (g == 0 && ctx->nmarks > 0 && !ctx->names[ctx->nmarks - 1]) --ctx->nmarks;
        if (st == RR_OK) st = cudaEventRecord(ctx->evLead[g], gs) == cudaSuccess ? RR_OK : fail(ctx, RR_ERR_CUDA, "record");
        prevSim = ctx->evSim[g];
        lo = hi;
        ++ng;
    }
    ctx->quiet = 1;
    if (st == RR_OK) {
        cudaStream_t rs = ctx->restStream;
        CUDA_TRY(cudaStreamWaitEvent(rs, ctx->evStart, 0));
        if (plan) st = launch_plan(ctx, ctx->d_pinst + lo, ctx->d_ws + lo, count - lo, max_side, rs, pflags);
        if (st == RR_OK)
            st = launch_batch(ctx, ctx->d_pinst + lo, ctx->d_ws + lo, count - lo, max_side, rs, SIM_CLASSES, prevSim,
                              nullptr);
        if (st == RR_OK) st = cudaEventRecord(ctx->evRest, rs) == cudaSuccess ? RR_OK : fail(ctx, RR_ERR_CUDA, "record");
    }
    ctx->quiet = 0;
    if (st != RR_OK) return st;
    for (int g = 0; g < ng; ++g) CUDA_TRY(cudaStreamWaitEvent(stream, ctx->evLead[g], 0));
    CUDA_TRY(cudaStreamWaitEvent(stream, ctx->evRest, 0));
    mark(ctx, stream, "k_scatter");
    k_scatter<<<(count + 255) / 256, 256, 0, stream>>>(d_inst, ctx->d_perm, ctx->d_pinst, count);
    mark(ctx, stream, nullptr);
    CUDA_TRY(cudaGetLastError());
    ctx->nlaunch += 3;
    return RR_OK;
}

extern "C" int rr_plan_batched(rr_ctx *ctx, rr_instance *d_inst, int count, int max_side, int flags,
                               cudaStream_t stream)
{
    if (!ctx || !d_inst || count < 1 || count > 65535 || max_side < 1 || max_side > RR_MAX_SIDE ||
        (flags & ~(RR_WITH_BATCH | RR_BATCH_ONLY | RR_GRAPH | RR_BIRD | RR_STRICT_RESERVOIR)))
        return fail(ctx, RR_ERR_ARG, "rr_plan_batched: bad argument (count=%d max_side=%d flags=%d)", count,
                    max_side, flags);
    int st = ensure_ws(ctx, count);
    if (st != RR_OK) return st;
    ctx->nmarks = 0;
    if (!(flags & RR_GRAPH)) return launch_sequence(ctx, d_inst, count, max_side, flags, stream);

    if (!(ctx->graph && ctx->gInst == d_inst && ctx->gCount == count && ctx->gMaxSide == max_side &&
          ctx->gFlags == flags)) {
        // capture on the context's own stream (the caller's may be the legacy
        // default stream, which cannot be captured); nothing runs yet
        drop_graph(ctx);
        const int64_t before = ctx->nlaunch;
        CUDA_TRY(cudaStreamBeginCapture(ctx->capStream, cudaStreamCaptureModeThreadLocal));
        ctx->capturing = 1;
        st = launch_sequence(ctx, d_inst, count, max_side, flags, ctx->capStream);
        ctx->capturing = 0;
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(ctx->capStream, &g);
        if (st == RR_OK && e != cudaSuccess)
            st = fail(ctx, RR_ERR_CUDA, "rr_plan_batched: graph capture: %s", cudaGetErrorString(e));
        if (st == RR_OK) {
            const cudaError_t e2 = cudaGraphInstantiate(&ctx->graph, g, cudaGraphInstantiateFlagUseNodePriority);
            if (e2 != cudaSuccess) {
                ctx->graph = nullptr;
                st = fail(ctx, RR_ERR_CUDA, "rr_plan_batched: graph instantiate: %s", cudaGetErrorString(e2));
            }
        }
        if (g) cudaGraphDestroy(g);
        ctx->gLaunches = ctx->nlaunch - before;
        ctx->nlaunch = before;
        if (st != RR_OK) {
            cudaGetLastError();
            return st;
        }
        ctx->gInst = d_inst; ctx->gCount = count; ctx->gMaxSide = max_side; ctx->gFlags = flags;
    }
    CUDA_TRY(cudaGraphLaunch(ctx->graph, stream));
    ctx->nlaunch += ctx->gLaunches;
    return RR_OK;
}

// One configuration's time for rr_autotune: the best of two runs of the
// call's launch sequence, or with RR_GRAPH the best of two replays of the
// graph captured under that configuration.
static int tune_time(rr_ctx *ctx, rr_instance *d_inst, int count, int max_side, int flags, cudaStream_t stream,
                     cudaEvent_t a, cudaEvent_t b, float *best)
{
    int st = RR_OK;
    *best = 1e30f;
    if (flags & RR_GRAPH) {
        drop_graph(ctx);
        st = rr_plan_batched(ctx, d_inst, count, max_side, flags, stream);      // capture, then the first replay
    }
    for (int rep = 0; rep < 2 && st == RR_OK; ++rep) {
        cudaEventRecord(a, stream);
        st = (flags & RR_GRAPH) ? rr_plan_batched(ctx, d_inst, count, max_side, flags, stream)
                                : launch_sequence(ctx, d_inst, count, max_side, flags, stream);
        cudaEventRecord(b, stream);
        if (st == RR_OK && cudaEventSynchronize(b) != cudaSuccess)
            st = fail(ctx, RR_ERR_CUDA, "rr_autotune: %s", cudaGetErrorString(cudaGetLastError()));
        float ms = 0.f;
        if (st == RR_OK && cudaEventElapsedTime(&ms, a, b) == cudaSuccess) *best = std::min(*best, ms);
    }
    return st;
}

extern "C" int rr_autotune(rr_ctx *ctx, rr_instance *d_inst, int count, int max_side, int flags,
                           cudaStream_t stream, int32_t *nclass, int32_t *shift, int32_t *pipe)
{
    if (!ctx || !d_inst || count < 1 || count > 65535 || max_side < 1 || max_side > RR_MAX_SIDE ||
        (flags & ~(RR_WITH_BATCH | RR_BATCH_ONLY | RR_GRAPH | RR_BIRD | RR_STRICT_RESERVOIR)))
        return fail(ctx, RR_ERR_ARG, "rr_autotune: bad argument (count=%d max_side=%d flags=%d)", count, max_side,
                    flags);
    int st = ensure_ws(ctx, count);
    if (st != RR_OK) return st;
    static const int NC[3] = {2, 4, 8}, SH[3] = {-1, 0, 1};
    cudaEvent_t a = nullptr, b = nullptr;
    CUDA_TRY(cudaEventCreate(&a));
    if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return fail(ctx, RR_ERR_CUDA, "rr_autotune: event"); }
    const int tracing = ctx->tracing;
    ctx->tracing = 0;
    float best = 1e30f;
    int bestN = ctx->nclass, bestS = ctx->shift;
    for (int i = 0; i < 9 && st == RR_OK; ++i) {
        ctx->nclass = NC[i / 3];
        ctx->shift = SH[i % 3];
        float t = 1e30f;
        st = tune_time(ctx, d_inst, count, max_side, flags, stream, a, b, &t);
        if (t < best) { best = t; bestN = ctx->nclass; bestS = ctx->shift; }
    }
    // then the pipeline split under that configuration
    ctx->nclass = bestN;
    ctx->shift = bestS;
    int bestP = ctx->pipe;
    best = 1e30f;
    for (int i = 0; i < PIPE_SPLITS && st == RR_OK; ++i) {
        ctx->pipe = i;
        float t = 1e30f;
        st = tune_time(ctx, d_inst, count, max_side, flags, stream, a, b, &t);
        if (t < best) { best = t; bestP = ctx->pipe; }
    }
    ctx->pipe = bestP;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    ctx->tracing = tracing;
    ctx->nclass = bestN;
    ctx->shift = bestS;
    drop_graph(ctx);                     // captured under another configuration
    if (nclass) *nclass = bestN;
    if (shift) *shift = bestS;
    if (pipe) *pipe = bestP;
    return st;
}

extern "C" int rr_set_config(rr_ctx *ctx, int nclass, int shift, int pipe)
{
    if (!ctx || nclass < 1 || nclass > rr_ctx::MAXCLASS || shift < -3 || shift > 3 || pipe < 0 || pipe >= PIPE_SPLITS)
        return fail(ctx, RR_ERR_ARG, "rr_set_config: bad argument (nclass=%d shift=%d pipe=%d)", nclass, shift, pipe);
    ctx->nclass = nclass;
    ctx->shift = shift;
    ctx->pipe = pipe;
    drop_graph(ctx);
    return RR_OK;
}

// Library-internal: size a context's descriptor table for `count` instances
// up front (the server does this before any wave so that no call allocates).
int rr_internal_reserve(rr_ctx *ctx, int count) { return ensure_ws(ctx, count); }

extern "C" int rr_debug_guard_limit(int64_t limit)
{
    if (limit < 0) return fail(nullptr, RR_ERR_ARG, "rr_debug_guard_limit: negative limit");
    int st = guard_cap_plan(limit);
    if (st == RR_OK) st = guard_cap_batch(limit);
    if (st == RR_OK) st = guard_cap_one(limit);
    return st == RR_OK ? RR_OK : fail(nullptr, st, "rr_debug_guard_limit: %s", cudaGetErrorString(cudaGetLastError()));
}

extern "C" int rr_set_tracing(rr_ctx *ctx, int enable)
{
    if (!ctx) return RR_ERR_ARG;
    ctx->tracing = enable != 0;
    ctx->nmarks = 0;
    return RR_OK;
}

extern "C" int rr_stage_times(rr_ctx *ctx, float *ms, const char **names, int cap)
{
    if (!ctx || cap < 0 || (cap > 0 && (!ms || !names))) return fail(ctx, RR_ERR_ARG, "rr_stage_times: bad argument");
    int n = 0;
    for (int i = 0; i + 1 < ctx->nmarks && n < cap; ++i) {
        if (!ctx->names[i]) continue;                 // end-of-sequence marker
        CUDA_TRY(cudaEventSynchronize(ctx->marks[i + 1]));
        float t = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&t, ctx->marks[i], ctx->marks[i + 1]));
        ms[n] = t;
        names[n] = ctx->names[i];
        ++n;
    }
    return n;
}
