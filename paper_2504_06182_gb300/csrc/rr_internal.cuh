// rr_internal.cuh -- device-side types and helpers shared by the kernels of
// the red-rec planner and batching routine (arXiv 2504.06182, Alg. 1 and 2).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "rr.h"

namespace rrk {

constexpr unsigned FULL = 0xffffffffu;

// Block coordinates of a stage (the stage functions of rr_plan.cuh,
// rr_bird.cuh and rr_batch.cuh): the hardware's when a stage runs as a
// kernel of its own; x = 0, gx = 1 when one block runs the whole path of one
// grid (the single-grid kernel), so that every grid-stride loop covers all
// of its items.
struct Blk { int x, y, gx; };
__device__ __forceinline__ Blk hw_blk() { return Blk{(int)blockIdx.x, (int)blockIdx.y, (int)gridDim.x}; }

// Column classification after the column phase (Alg. 1 first loop, solved for
// every column of non-negative surplus at once as in Sec. III.D).
enum ColKind : int32_t {
    KIND_TARGET_SOLVED = 0,   // target column, surplus >= 0: exact 1D window solve
    KIND_RECEIVER = 1,        // target column, surplus < 0
    KIND_OUTER_FULL = 2,      // outside the target columns, enough atoms to fill its reservoir cells
    KIND_OUTER_PART = 3       // outside the target columns, fewer atoms than reservoir cells
};

struct ColInfo {
    int32_t K, ntop, nband, nbot;   // atoms: all, rows < r0, rows in [r0, r1), rows >= r1
    int32_t sigma;                  // surplus after the column phase
    int32_t kind;
    int32_t ptop, pbot;             // donatable pool sizes (nearest-to-band first)
    int32_t tbase, bbase;           // atom index of the nearest top / bottom pool atom
    int32_t a;                      // target solved: top atoms taken into the window
    int32_t kd_end, ku_start;       // solve order ranges (see emission)
    int32_t nmoves;                 // moves of this column's column-phase unit
    int32_t topRun, botRun;         // outer full: atoms already on their virtual targets
};

// One pairing iteration (Alg. 1 main loop).
struct Event {
    int32_t kase;       // 1: receiver saturated, 2: both saturated, 3: donor exhausted (delayed)
    int32_t i, j;       // donor, receiver
    int32_t x, a;       // tokens exchanged, of which a come from above the band
    int32_t t0, b0;     // donor pool cursors (nearest-first index) before the exchange
    int32_t next;       // next event with the same receiver, -1
};

// A receiver unit, in the order receivers become saturated.
struct RecvInfo {
    int32_t j;
    int32_t ev_first;   // first event whose receiver is j (linked by Event::next)
    int32_t ncontrib;   // events in that list
    int32_t nT;         // sources above the band (mandatory + chosen)
    int32_t kd_end, ku_start, nmoves;
    int32_t pad;
};

struct Arena {
    char *base;
    unsigned long long size;
    unsigned long long *top;   // device bump pointer
};

struct JobWS {
    // planning
    uint32_t *colbits;     // n * W, column-major bit columns (bit r & 31 of word r >> 5)
    int16_t *atomRows;     // n * m: rows of the atoms of each column, ascending
    int16_t *holeRows;     // n * h: rows of the empty band traps of each column, ascending
    ColInfo *col;          // n
    RecvInfo *recv;        // n
    Event *ev;             // n + 1
    int32_t *unitOff;      // 2n + 1
    int32_t nrecv, nev;
    // batching (Gamma + simulation)
    int64_t P;             // total path vertices (sum of path length + 1)
    int32_t *pairOff;      // k + 1
    int32_t *nextAt;       // P
    int32_t *succCnt;      // k: distinct successors of each path
    int32_t *succ;         // P: a path's successors at its vertex offset (pairOff)
    int32_t *indeg;        // k
    int4 *rec;             // k: packed geometry, successor count, overflow offset
    int4 *succ4;           // k: first four successors (flagged, -1 padded)
    int32_t *ready0;       // k + 1: moves without predecessors; [k] = their count
    // Gamma by sweeps: moves ending in each column, L-moves starting on each row
    int32_t *colOff, *colCur, *colList;   // n + 1, n, k
    int32_t *rowOff, *rowCur, *rowList;   // m + 1, m, k
    int32_t *firstH;       // m * n: lowest-id L-move crossing each vertex, -1
    void *slotOvf;         // k simulation slots beyond the shared-memory ones
    int32_t *ovfFree;      // k: recycled overflow slots
    // path-vertex offsets by the multi-block scan (large move lists only):
    // one status word per tile, the tile counter
    unsigned long long *lbStatus;
    int32_t *lbCounter;
};

// Multi-block single-pass scan (decoupled look-back) of the path-vertex
// offsets: tiles of LB_TILE moves, taken in order from a per-instance
// counter by blocks of LB_THREADS threads; used for move lists of at least
// LB_MIN_MOVES (below that one block scans them).
constexpr int LB_THREADS = 512, LB_ITEMS = 8, LB_TILE = LB_THREADS * LB_ITEMS;
constexpr int64_t LB_MIN_MOVES = 1 << 16;

// Side bound of simulation size class c of nclass over grids up to
// max_side (the last class takes max_side itself).
__host__ __device__ inline int class_side(int max_side, int c, int nclass)
{
    if (c >= nclass - 1) return max_side;
    const int s = (max_side * (c + 1) + nclass - 1) / nclass;
    return s < 32 ? 32 : s;
}

// Shared memory of one batching-simulation block (one warp, one instance):
// sort / merge buffer, slot table, id map, members, successor buffer,
// pickup bitmaps, list links and heads (ix bytes each), step counters and
// the free-slot stack. The kernel's layout follows this order.
constexpr int MAPN = 256;       // id -> slot cache for finding the next leader
constexpr int SBUF = 256;       // successor entries released per round
__host__ __device__ inline size_t sim_smem_bytes(int slotCap, int lineCap, int ix)
{
    const size_t S = (size_t)slotCap, L = (size_t)lineCap;
    return 8 * 2 * (L + 2) +                                            // Kb
           4 * (2 * S + MAPN + 2 * (L + 2) + SBUF + 4 * ((L + 31) / 32)) +  // key id, map, Mid Msl, sbuf, bits
           (size_t)ix * (4 * S + 8 * L) +                                // rp rn cp cn, row and column heads
           2 * 4 * S +                                                   // t, legEnd, dstRow, free stack
           64;
}

// Status of an instance between the two simulation passes: the narrow pass
// (shared-memory slots only) ran out of slots and the wide pass redoes it.
// The wide pass always follows in the same launch sequence, so callers never
// see it.
constexpr int32_t RR_SIM_RETRY = 100;

// Successor entries carry this flag when the successor has a single
// predecessor: it becomes ready as soon as that predecessor finishes.
constexpr int32_t SUCC_SINGLE = 1 << 30;
constexpr int32_t SUCC_ID = SUCC_SINGLE - 1;

__device__ __forceinline__ void *arena_alloc(const Arena &A, unsigned long long bytes, bool *ok)
{
    bytes = (bytes + 255ull) & ~255ull;
    unsigned long long off = atomicAdd(A.top, bytes);
    if (off + bytes > A.size) { *ok = false; return nullptr; }
    return A.base + off;
}

__device__ __forceinline__ int warp_incl_scan(int v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

__device__ __forceinline__ int warp_sum(int v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        unsigned long long u = __shfl_xor_sync(FULL, v, o);
        v = u > v ? u : v;
    }
    return v;
}

// Bits of rows [lo, hi) that fall in word w (rows 32w .. 32w+31).
__device__ __forceinline__ uint32_t row_mask(int w, int lo, int hi)
{
    int a = max(lo - 32 * w, 0), b = min(hi - 32 * w, 32);
    if (b <= a) return 0u;
    uint32_t hiMask = b >= 32 ? FULL : ((1u << b) - 1u);
    uint32_t loMask = (1u << a) - 1u;
    return hiMask & ~loMask;
}

__device__ __forceinline__ int iabs(int v) { return v < 0 ? -v : v; }
__device__ __forceinline__ int isgn(int v) { return (v > 0) - (v < 0); }

// Direction codes of rr_op.
__device__ __forceinline__ int step_dir(int sr, int sc, int dr, int dc, int t)
{
    int hl = iabs(dc - sc);
    if (t < hl) return dc > sc ? 3 : 2;
    return dr > sr ? 1 : 0;
}

__device__ __forceinline__ void path_cell(int sr, int sc, int dr, int dc, int t, int *r, int *c)
{
    int hl = iabs(dc - sc);
    if (t <= hl) { *r = sr; *c = sc + t * isgn(dc - sc); }
    else { *r = sr + (t - hl) * isgn(dr - sr); *c = dc; }
}

// Test hook: when positive, the pairing loop and the batching simulation
// stop after this many iterations with RR_ERR_TIMEOUT, as when their own
// bounds run out (rr_debug_guard_limit sets it in every module that runs
// them). Zero keeps the built-in bounds.
static __device__ long long g_guard_cap = 0;

// Status helpers: an instance is live while its status is RR_OK.
__device__ __forceinline__ void set_status(rr_instance *I, int st)
{
    atomicCAS(&I->status, 0, st);
}
__device__ __forceinline__ bool live(const rr_instance *I) { return I->status == RR_OK; }

// Adds a warp's elementary-step count to the instance total (every lane of
// the warp calls it).
__device__ __forceinline__ void add_steps(rr_instance *I, long long v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd((unsigned long long *)&I->n_steps, (unsigned long long)v);
}

// Largest a in [lo, hi] with a == lo or delta(a) <= 0, for a non-decreasing
// delta (the discrete derivative of a convex cost). Warp-cooperative: every
// round probes 32 evenly spaced candidates.
template <class F>
__device__ int split_search(int lo, int hi, F delta)
{
    const int lane = threadIdx.x & 31;
    for (int guard = 0; hi > lo && guard < 8; ++guard) {
        const int span = hi - lo;
        const int al = lo + (int)(((long long)(lane + 1) * span + 31) / 32);
        const bool ok = delta(al) <= 0;
        const unsigned bal = __ballot_sync(FULL, ok);
        if (bal == 0u) {
            hi = __shfl_sync(FULL, al, 0) - 1;
        } else {
            const int L = 31 - __clz(bal);
            const int aL = __shfl_sync(FULL, al, L);
            const int aN = __shfl_sync(FULL, al, L < 31 ? L + 1 : 31);
            lo = aL;
            if (L < 31) hi = aN - 1;
        }
    }
    return lo;
}

// Number of band atoms i of a target column with (b_i - i) <= T, i.e. with at
// most T - r0 empty band traps above them. hr: the column's band holes.
__device__ __forceinline__ int band_P(const int16_t *hr, int nh, int nband, int r0, int T)
{
    const int u = T - r0;
    if (u < 0) return 0;
    if (u >= nh) return nband;
    return (int)hr[u] - r0 - u;
}

} // namespace rrk

// Library-internal hooks between translation units (not part of the C ABI).
int rr_internal_reserve(rr_ctx *ctx, int count);

namespace rrk {
// Per-module setters of g_guard_cap (rr_plan.cu, rr_batch.cu, rr_one.cu).
int guard_cap_plan(long long cap);
int guard_cap_batch(long long cap);
int guard_cap_one(long long cap);
// The single-grid kernel (rr_one.cu): one block of ONE_THREADS threads runs
// planning, Gamma and batching of one grid with sides up to ONE_MAX_SIDE.
constexpr int ONE_THREADS = 256;
constexpr int ONE_MAX_SIDE = 256;
size_t one_smem_bytes(int side, int flags);
const void *one_kernel();
int one_launch(rr_instance h, rr_instance *d_inst, JobWS *d_ws, Arena A, int flags, int side, size_t smem,
               rr_instance *hostOut, cudaStream_t s);
} // namespace rrk
