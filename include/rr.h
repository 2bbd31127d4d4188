/*
 * rr.h -- C ABI of the GB300 red-rec planner and batching routine.
 *
 * Method: Afiouni et al., "Efficient algorithms to solve atom reconfiguration
 * problems III" (arXiv 2504.06182): the improved red-rec algorithm (Alg. 1,
 * Sec. III.C, executed in the column order of the parallel variant of Sec.
 * III.D) and the batching routine (Alg. 4 with the local constraint set of
 * Sec. IV). All arithmetic is integer.
 *
 * Memory: every buffer argument named d_* is caller-owned memory the device
 * can address, normally device memory; the library never frees or retains it.
 * Output buffers may also be host memory mapped for the device (pinned with
 * cudaHostAlloc / cudaHostRegister): the kernels then write the results
 * straight into host memory, with no separate copy. The batching kernels read
 * the move list several times, so it is best kept in device memory; batches
 * and members are only written. Host pointers (n_moves, n_ops, ...) are
 * written before the call returns. Workspace lives in the context.
 * Streams: work is issued on `stream`; calls that return counts to host
 * pointers synchronise that stream before returning.
 * Errors: every entry point returns an rr_status; no CPU fallback exists and
 * nothing fails silently. On RR_ERR_CAPACITY the required sizes are written to
 * the count pointers and no output element is valid.
 * Limits: 1 <= m, n <= RR_MAX_SIDE.
 */
#ifndef RR_H
#define RR_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RR_MAX_SIDE 1024

typedef enum {
    RR_OK = 0,
    RR_INFEASIBLE = 1,       /* total surplus negative: no plan, zero moves (Sec. III.C) */
    RR_ERR_ARG = -1,         /* bad argument (sizes, rectangle, null pointers, layout) */
    RR_ERR_CAPACITY = -2,    /* an output buffer is too small; required sizes returned */
    RR_ERR_CUDA = -3,        /* a CUDA runtime call failed */
    RR_ERR_TIMEOUT = -4,     /* a bounded device loop hit its iteration limit */
    RR_ERR_WORKSPACE = -5,   /* the context's device arena is too small */
    RR_ERR_INTERNAL = -6     /* a device-side invariant check failed */
} rr_status;

typedef enum { RR_U8 = 0, RR_BITS32 = 1 } rr_layout;

/* Target rectangle: rows [r0, r1), columns [c0, c1), half-open,
 * 0 <= r0 < r1 <= m, 0 <= c0 < c1 <= n. */
typedef struct { int32_t r0, c0, r1, c1; } rr_rect;

/* One move = one extraction-displacement-implantation cycle along a shortest
 * path (Sec. II.A-C): along row src_row from src_col to dst_col, then along
 * column dst_col from src_row to dst_row. */
typedef struct { int32_t src_row, src_col, dst_row, dst_col; } rr_move;

/* One batch of Alg. 4: members[first .. first+count) are the ids (indices into
 * the move list) of the moves whose tokens advance one elementary step in
 * direction dir: 0 = row-1, 1 = row+1, 2 = column-1, 3 = column+1. */
typedef struct { int32_t dir, first, count; } rr_op;

typedef struct rr_ctx rr_ctx;

/* Context: owns the device workspace arena (bytes; 0 = default 1 GiB) on the
 * current CUDA device. Not thread-safe: one host thread per context. */
int rr_ctx_create(rr_ctx **ctx, int64_t arena_bytes);
int rr_ctx_destroy(rr_ctx *ctx);

/* Plan one grid (Alg. 1). Grid layout: RR_U8 = m*n bytes row-major, 0/1;
 * RR_BITS32 = m rows of ceil(n/32) uint32 words, bit (c & 31) of word (c >> 5)
 * is trap c, least significant bit first. Moves are emitted in execution
 * order: column-phase units in column order, then receiver units in the order
 * the receivers become saturated; inside a unit, paths toward larger rows by
 * descending target row, then paths toward smaller rows by ascending target
 * row (Sec. III.A). cap = capacity of d_moves in moves. Writes *n_moves
 * (required count on RR_ERR_CAPACITY; 0 on RR_INFEASIBLE). Synchronises. */
int rr_plan(rr_ctx *ctx, const void *d_grid, int layout, int m, int n, rr_rect rect,
            rr_move *d_moves, int64_t cap, int64_t *n_moves, cudaStream_t stream);

/* Plan one grid with the bird algorithm (Alg. 2, Sec. III.E). Arguments,
 * layouts, output and synchronisation as rr_plan. The column phase is
 * rr_plan's (the same moves, first); then the columns of negative surplus are
 * filled one by one, left to right, each through its generalised 1D instance:
 * the column's own atoms plus every atom in a reservoir row (a row outside
 * [r0, r1)) of every other column, an atom at column distance d standing on
 * vertex row - d (above the band) or row + d (below it) of the column. The
 * tokens of least total distance are taken (a vertex holding several gives
 * its nearest columns' tokens, left before right), matched in order and
 * emitted as one unit with rr_plan's order inside a unit. The paper states
 * bird for centred targets; nothing here needs the centring. Feasibility is
 * rr_plan's (RR_INFEASIBLE iff the total surplus is negative). */
int rr_bird_plan(rr_ctx *ctx, const void *d_grid, int layout, int m, int n, rr_rect rect,
                 rr_move *d_moves, int64_t cap, int64_t *n_moves, cudaStream_t stream);

/* rr_plan / rr_bird_plan with explicit planning flags: RR_BIRD selects the
 * bird algorithm; RR_STRICT_RESERVOIR selects the strict reading of target
 * sub-rectangles. By default (the reading this library uses elsewhere) a
 * column outside [c0, c1) with at least m - (r1 - r0) atoms is first solved
 * on its own with its reservoir traps (rows outside [r0, r1)) as targets, so
 * that its band-row atoms become donatable; with RR_STRICT_RESERVOIR such
 * columns stay as they are and donate only the atoms already in their
 * reservoir rows (Sec. III.C: donors give reservoir atoms only), so every
 * atom moves at most once, at the price of feasibility (most centred square
 * targets of 0.7 times the side at fill 0.6 become infeasible). With c0 = 0
 * and c1 = n both readings are the paper's algorithm. Other arguments and
 * behaviour as rr_plan; unknown flags give RR_ERR_ARG. */
int rr_plan_mode(rr_ctx *ctx, const void *d_grid, int layout, int m, int n, rr_rect rect, int flags,
                 rr_move *d_moves, int64_t cap, int64_t *n_moves, cudaStream_t stream);

/* Batch a move list (Alg. 4 + Sec. IV): dependencies = every earlier move
 * whose path shares a vertex; ready moves are visited in ascending id and a
 * move's next step joins the batch iff it has the first member's direction and
 * its token shares a row or a column with every member's token. d_moves must
 * be an unobstructed ordered path system on an m x n grid (e.g. rr_plan's
 * output). Writes *n_ops and *n_members (= total elementary steps).
 * Synchronises. */
int rr_batch(rr_ctx *ctx, const rr_move *d_moves, int64_t n_moves, int m, int n,
             rr_op *d_ops, int64_t cap_ops, int32_t *d_members, int64_t cap_members,
             int64_t *n_ops, int64_t *n_members, cudaStream_t stream);

/* Plan one grid and, with RR_WITH_BATCH, batch its moves in ONE kernel
 * launch: one block runs every stage of rr_plan (or rr_bird_plan with
 * RR_BIRD) and of rr_batch in turn, with block barriers instead of kernel
 * boundaries, no host round trip and one synchronisation. The paper's GPU
 * red-rec is a single kernel for this reason (Sec. III.D): the latency of one
 * reconfiguration cycle on one small grid, where launch gaps and host
 * round trips would dominate the multi-kernel path. Sides up to
 * RR_ONE_MAX_SIDE. flags: RR_WITH_BATCH, RR_BIRD, RR_STRICT_RESERVOIR (as
 * rr_plan_mode). Outputs as rr_plan (moves) and, with RR_WITH_BATCH, as
 * rr_batch (ops, members; ignored without it). counts (host, 4 entries):
 * n_moves, n_steps (total elementary steps), n_ops, n_members. Returns
 * RR_OK, RR_INFEASIBLE (no moves), RR_ERR_CAPACITY (the counts hold the
 * required sizes: exact for moves; n_ops, n_members = n_steps for batches,
 * an upper bound for n_ops) or an error. Results are bit-identical to
 * rr_plan_mode followed by rr_batch. Synchronises `stream`. */
#define RR_ONE_MAX_SIDE 256
int rr_plan_one(rr_ctx *ctx, const void *d_grid, int layout, int m, int n, rr_rect rect, int flags,
                rr_move *d_moves, int64_t cap_moves, rr_op *d_ops, int64_t cap_ops, int32_t *d_members,
                int64_t cap_members, int64_t *counts, cudaStream_t stream);

/* Many independent grids in one launch sequence (device-resident
 * descriptors). Inputs per instance: grid, layout, m, n, rect, output
 * pointers and capacities. Outputs per instance: status, n_moves, n_steps
 * (total elementary steps), and with RR_WITH_BATCH n_ops and n_members.
 * On RR_ERR_CAPACITY for an instance, its counts hold the required sizes
 * (n_ops is then an upper bound, = n_steps). The call itself returns RR_OK
 * when it issued the work (no synchronisation); read the per-instance status
 * after synchronising the stream. */
#define RR_WITH_BATCH 1
#define RR_BATCH_ONLY 2   /* skip planning: instances carry moves and n_moves (status RR_OK) */
#define RR_GRAPH 4        /* replay a captured CUDA graph of the launch sequence (below) */
#define RR_BIRD 8         /* plan with the bird algorithm (as rr_bird_plan) instead of red-rec */
#define RR_STRICT_RESERVOIR 16  /* strict reading of target sub-rectangles (rr_plan_mode) */
typedef struct {
    const void *grid;
    int32_t layout, m, n, pad0;
    rr_rect rect;
    rr_move *moves;     int64_t cap_moves;
    rr_op *ops;         int64_t cap_ops;
    int32_t *members;   int64_t cap_members;
    int64_t n_moves, n_steps, n_ops, n_members;   /* outputs */
    int32_t status, pad1;                         /* output */
} rr_instance;

/* With RR_BATCH_ONLY the planning kernels are skipped and each instance's
 * moves[0 .. n_moves) are batched as by rr_batch (status must be RR_OK).
 * count in [1, 65535]; max_side bounds m and n of every instance (an
 * instance above it gets RR_ERR_ARG); it sizes the launch shapes. The call
 * may grow the context's descriptor table (a synchronous cudaMalloc), so the
 * first call with a larger count must not be inside stream capture.
 * With RR_GRAPH the context captures the call's whole launch sequence (one
 * graph of all its kernels and memsets) the first time, on a stream of its
 * own, and afterwards launches that graph on `stream` for as long as
 * d_inst, count, max_side and flags stay the same; the descriptors and the
 * memory they point to may change between calls (the kernels read them on
 * the device). Any other call that grows the descriptor table drops the
 * graph. Stage tracing does not cover graph launches. Nothing in the paper
 * corresponds to this; it removes the per-call launch cost for callers that
 * re-plan the same set of buffers (a control loop, the bench). */
int rr_plan_batched(rr_ctx *ctx, rr_instance *d_inst, int count, int max_side, int flags,
                    cudaStream_t stream);

/* Launch-configuration autotuner for rr_plan_batched (nothing in the paper
 * corresponds to it). Runs the call's launch sequence on these instances,
 * timed with CUDA events on `stream` (best of two each): first under nine
 * configurations (2, 4 or 8 simulation size classes, times per-grid block
 * budgets of the planning and graph kernels scaled by 1/2, 1 or 2), then,
 * with the best of those, under five pipeline splits (see below): 0 none,
 * 1 the largest quarter first, 2 the largest 1/16 then up to 1/4, 3 groups
 * ending at 1/16, 1/8, 1/4 and 1/2, 4 groups ending at 1/64, 1/16 and 1/4. The fastest is kept in the context for
 * later rr_plan_batched calls (a captured RR_GRAPH graph is dropped) and
 * written to *nclass, *shift (log2 of the budget scale) and *pipe (the
 * split) when those are not NULL. Every
 * configuration computes the same results, so the descriptors and outputs
 * hold this call's results afterwards. Synchronises; flags as
 * rr_plan_batched. With RR_GRAPH each configuration is captured as a graph
 * and timed by its replays, so the choice suits later RR_GRAPH calls (the
 * fastest configuration for direct launches can replay a few percent slower
 * than another one).
 *
 * Pipeline (batched calls with batching over at least 256 grids): the grids
 * are ordered by side, largest first, into a descriptor copy; each leading
 * group is planned, given its conflict graph and simulated on a stream of
 * its own (priorities descending) while the rest is planned and given its
 * graphs on a low-priority stream; each group's simulations start once the
 * previous group's have started; per-grid outputs are then copied back into
 * the caller's descriptors. The default is split 1. */
int rr_autotune(rr_ctx *ctx, rr_instance *d_inst, int count, int max_side, int flags,
                cudaStream_t stream, int32_t *nclass, int32_t *shift, int32_t *pipe);

/* Sets the launch configuration of later rr_plan_batched calls directly (as
 * rr_autotune leaves it): nclass in [1, 8] simulation size classes, block
 * budgets scaled by 2^shift (shift in [-3, 3]), pipeline split pipe in
 * [0, 4] (as above). Drops a captured RR_GRAPH graph. Results do not depend
 * on the configuration. The defaults are nclass 4, shift 0, pipe 1. */
int rr_set_config(rr_ctx *ctx, int nclass, int shift, int pipe);

/* ------------------------------------------------------------------ serving
 * Continuous batching of planning requests (red-rec + batching per request):
 * a request is admitted as soon as its grid and its move list (room for
 * 2 m n moves, each atom moves at most twice) fit in the device input pool
 * and fewer than `slots` requests are resident (first come, first served), planned in waves (one rr_plan_batched call over the
 * requests admitted since the previous wave) on a pool of streams so that
 * waves overlap on the device, and, once a request's exact number of
 * elementary steps is known, given result memory from a device heap and
 * batched in a second wave (memory-based admission). A worker thread owned
 * by the server drives the pipeline; the calling threads only submit, poll
 * and release. Results stay on the device until released. Each stream has a
 * context of its own; a wave of at most 8 requests runs its simulation as
 * one launch on its stream. With many streams, start the process with
 * CUDA_DEVICE_MAX_CONNECTIONS=32 (read when CUDA initialises): with the
 * default 8 hardware work queues, waves on different streams wait behind
 * each other's long simulation kernels. */
typedef struct rr_server rr_server;
typedef struct {
    int32_t max_side;        /* largest m or n accepted, <= RR_MAX_SIDE */
    int32_t slots;           /* requests admitted and not yet released, at most */
    int32_t streams;         /* waves in flight at once */
    int32_t max_wave;        /* requests per wave, <= slots */
    int32_t flags;           /* RR_WITH_BATCH to also batch every plan; RR_BIRD to plan with bird;
                                RR_STRICT_RESERVOIR as in rr_plan_mode */
    int32_t pad;
    int64_t arena_bytes;     /* workspace arena per stream */
    int64_t heap_bytes;      /* device heap for batch results (16 B per elementary step) */
    int64_t input_bytes;     /* device pool for grids and move lists; 0: room for `slots`
                                requests of max_side */
} rr_serve_config;
typedef struct {
    int32_t status;          /* RR_OK, RR_INFEASIBLE or an error; RR_ERR_CAPACITY if the heap can never hold it */
    int32_t m, n, pad;
    int64_t n_moves, n_steps, n_ops, n_members;
    const rr_move *d_moves;  /* device results, valid until rr_serve_release */
    const rr_op *d_ops;
    const int32_t *d_members;
    double t_submit_us, t_admit_us, t_done_us;   /* host clock, microseconds since rr_serve_open */
} rr_serve_result;
/* Allocates every device buffer up front (slots, heap, arenas, descriptors). */
int rr_serve_open(rr_server **srv, const rr_serve_config *cfg);
/* Copies the grid (host memory, layouts as rr_plan) into the request queue
 * and returns a ticket at once. RR_ERR_ARG for sizes above max_side;
 * RR_ERR_CAPACITY if the grid and its move list could never fit the input
 * pool. */
int rr_serve_submit(rr_server *srv, const void *h_grid, int layout, int m, int n, rr_rect rect,
                    int64_t *ticket);
/* Waits up to timeout_us (0: just look) for the ticket: RR_OK and *out
 * filled when done, RR_ERR_TIMEOUT otherwise, RR_ERR_ARG for an unknown
 * ticket. */
int rr_serve_poll(rr_server *srv, int64_t ticket, rr_serve_result *out, int64_t timeout_us);
/* Frees the ticket's slot and result memory (its device pointers die). */
int rr_serve_release(rr_server *srv, int64_t ticket);
/* Stops the worker after in-flight waves finish and frees everything. */
int rr_serve_close(rr_server *srv);

/* rr_plan without allocation, for callers that must not allocate device
 * memory: a real-time reconfiguration loop (cudaMalloc/cudaFree can
 * synchronise the device and take unbounded time between imaging and the
 * tweezer moves), or a plug-in whose device memory belongs to another
 * allocator. The paper has no counterpart; the arguments, outputs and return
 * codes are those of rr_plan, and no context is used.
 * Workspace: a file-scope device array of RR_NOALLOC_SCRATCH_BYTES that every
 * GPU loading the library holds until exit. Grids above RR_NOALLOC_MAX_SIDE
 * in either side are rejected with RR_ERR_ARG. The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress): make that first
 * call before any stream capture. All calls share the array and it keeps
 * the last call's contents: calls that overlap on the GPU (other streams,
 * other host threads) race and must be serialised by the caller.
 * The call copies the move count back into host memory and synchronises
 * `stream` before returning; on a stream that is being captured it returns
 * RR_ERR_ARG without enqueuing anything. */
#define RR_NOALLOC_MAX_SIDE 256
#define RR_NOALLOC_SCRATCH_BYTES (512 * 1024)
int rr_plan_noalloc(const void *d_grid, int layout, int m, int n, rr_rect rect,
                    rr_move *d_moves, int64_t cap, int64_t *n_moves, cudaStream_t stream);

/* Stage tracing. With tracing on, every public call records a CUDA event on
 * its stream before each kernel and after the last one. rr_stage_times then
 * waits for those events and writes, for the most recent call, each kernel's
 * name (static strings) and elapsed milliseconds; it returns the number of
 * stages written (at most cap) or a negative rr_status. */
int rr_set_tracing(rr_ctx *ctx, int enable);
int rr_stage_times(rr_ctx *ctx, float *ms, const char **names, int cap);

/* Test hook for the failure path (nothing in the paper corresponds to it):
 * with limit > 0 the pairing loop of the planner (Alg. 1) and the batching
 * simulation (Alg. 4) stop after `limit` iterations and report
 * RR_ERR_TIMEOUT, exactly as when their built-in iteration bounds run out, so
 * that a test can drive that path without a fault; limit 0 restores the
 * built-in bounds. It holds for every context of the process on the current
 * device; not for production use. Returns RR_ERR_ARG for a negative limit. */
int rr_debug_guard_limit(int64_t limit);

/* Kernels this context has launched since it was created (every public call
 * adds the launches it made; the size-class simulation counts one launch per
 * class). For accounting only: reading it does not synchronise. Returns
 * RR_ERR_ARG for a null argument. */
int rr_launch_count(rr_ctx *ctx, int64_t *launches);

/* Last error text of this context; with ctx NULL, of the calling thread's
 * last call that had no context (e.g. a failed rr_ctx_create). Never NULL;
 * valid until the next call on the same context or thread. */
const char *rr_last_error(rr_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif
