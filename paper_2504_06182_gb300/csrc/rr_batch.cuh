// rr_batch.cuh -- stages of the batching routine (arXiv 2504.06182, Alg. 4 with the
// local constraint set of Sec. IV) on the GPU.
//
// Gamma (Sec. IV, "Input to the batching routine"): move b depends on every
// earlier move whose path shares a vertex with it. It is enough to keep, for
// every vertex, the immediately preceding path through it; a move is ready
// once all of those have finished. The kernels below build, per vertex, the
// list of paths through it in id order, and from it the de-duplicated
// successor lists and in-degrees.
//
// Alg. 4 itself runs as an event-driven simulation, one warp per instance.
// The lowest-id unfinished move is always ready (nothing earlier is
// unfinished), so it is always the first member ("leader") of the batch. With
// the leader's token at (r, c) moving in direction d, the other members are
// the ready moves stepping in direction d whose tokens lie on row r (set A)
// or on column c (set B): the one of A and B holding the smaller id wins,
// because pairwise row-or-column sharing with three or more tokens forces
// them onto one line. While the members advance together the batch can only
// change when a member turns or finishes, or when the leader's row (vertical
// d) or column (horizontal d) reaches a waiting ready move of direction d.
// Between such events every batch is the same, so runs of identical batches
// are written in one go.
#include <type_traits>
#pragma once
#include "rr_internal.cuh"

namespace rrk {

// Chunked block-wide exclusive scan of v[0..len) in place; returns the total.
// Every thread of the block must call it.
__device__ inline long long block_exclusive_scan(int32_t *v, int len, long long *s_tmp /* >= 33 */)
{
    const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int per = (len + T - 1) / T;
    const int lo = min(len, tid * per), hi = min(len, lo + per);
    long long sum = 0;
    for (int i = lo; i < hi; ++i) sum += v[i];
    long long incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long u = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) s_tmp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        long long w = lane < (T >> 5) ? s_tmp[lane] : 0;
        long long wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long u = __shfl_up_sync(FULL, wi, o);
            if (lane >= o) wi += u;
        }
        if (lane < (T >> 5)) s_tmp[lane] = wi - w;
        if (lane == 31) s_tmp[32] = wi;
    }
    __syncthreads();
    long long run = s_tmp[wid] + incl - sum;
    for (int i = lo; i < hi; ++i) { const long long x = v[i]; v[i] = (int32_t)run; run += x; }
    const long long total = s_tmp[32];
    __syncthreads();
    return total;
}

// ----------------------------------------------------------- set-up pass
// One block per instance: check the moves, count path vertices, allocate.
__device__ inline void s_bsetup(const Blk B, rr_instance *inst, JobWS *wsv, int count, Arena A, int lookback)
{
    __shared__ long long s_tmp[34];
    __shared__ int s_bad;
    const int q = B.x;
    if (q >= count) return;
    rr_instance *I = &inst[q];
    if (!live(I)) return;
    JobWS &ws = wsv[q];
    const int m = I->m, n = I->n;
    const int64_t k = I->n_moves;
    if (lookback && k >= LB_MIN_MOVES) {
        // a large move list: checking the moves, counting their vertices and
        // the offsets are the work of the multi-block k_pairoff_lookback,
        // which also allocates the vertex-sized arrays once the total is
        // known; here only the move-sized arrays
        __shared__ int s_ok;
        if (threadIdx.x == 0) {
            bool ok = k <= 0x3fffffff;
            const unsigned long long cells = (unsigned long long)m * n;
            if (!ok) I->status = RR_ERR_ARG;
            ws.P = -1;
            ws.pairOff = (int32_t *)arena_alloc(A, 4ull * (k + 1), &ok);
            ws.colOff = (int32_t *)arena_alloc(A, 4ull * (n + 1), &ok);
            ws.colCur = (int32_t *)arena_alloc(A, 4ull * (n + 1), &ok);
            ws.colList = (int32_t *)arena_alloc(A, 4ull * (k + 1), &ok);
            ws.rowOff = (int32_t *)arena_alloc(A, 4ull * (m + 1), &ok);
            ws.rowCur = (int32_t *)arena_alloc(A, 4ull * (m + 1), &ok);
            ws.rowList = (int32_t *)arena_alloc(A, 4ull * (k + 1), &ok);
            ws.firstH = (int32_t *)arena_alloc(A, 4ull * cells, &ok);
            ws.succCnt = (int32_t *)arena_alloc(A, 4ull * (k + 1), &ok);
            ws.indeg = (int32_t *)arena_alloc(A, 4ull * (k + 1), &ok);
            ws.rec = (int4 *)arena_alloc(A, 32ull * (k + 1), &ok);
            ws.succ4 = ws.rec + 1;
            ws.ready0 = (int32_t *)arena_alloc(A, 4ull * (k + 1) + 16, &ok);
            ws.slotOvf = arena_alloc(A, 40ull * (k + 1), &ok);
            ws.ovfFree = (int32_t *)arena_alloc(A, 4ull * (k + 1), &ok);
            ws.nextAt = nullptr;
            ws.succ = nullptr;
            ws.lbStatus = (unsigned long long *)arena_alloc(A, 8ull * ((k + LB_TILE - 1) / LB_TILE), &ok);
            ws.lbCounter = (int32_t *)arena_alloc(A, 4, &ok);
            if (!ok && live(I)) I->status = RR_ERR_WORKSPACE;
            s_ok = live(I);
        }
        __syncthreads();
        if (!s_ok) return;
        for (int64_t t = threadIdx.x; t < (k + LB_TILE - 1) / LB_TILE; t += blockDim.x) ws.lbStatus[t] = 0ull;
        if (threadIdx.x == 0) { *ws.lbCounter = 0; ws.ready0[k] = 0; }
        for (int c = threadIdx.x; c <= n; c += blockDim.x) { ws.colOff[c] = 0; ws.colCur[c] = 0; }
        for (int r = threadIdx.x; r <= m; r += blockDim.x) { ws.rowOff[r] = 0; ws.rowCur[r] = 0; }
        return;
    }
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    long long P = 0, steps = 0;
    for (int64_t b = threadIdx.x; b < k; b += blockDim.x) {
        const rr_move p = I->moves[b];
        if (p.src_row < 0 || p.src_row >= m || p.dst_row < 0 || p.dst_row >= m || p.src_col < 0 ||
            p.src_col >= n || p.dst_col < 0 || p.dst_col >= n || (p.src_row == p.dst_row && p.src_col == p.dst_col))
            s_bad = 1;
        const int len = iabs(p.dst_col - p.src_col) + iabs(p.dst_row - p.src_row);
        steps += len; P += len + 1;
    }
    for (int o = 16; o; o >>= 1) {
        P += __shfl_xor_sync(FULL, P, o);
        steps += __shfl_xor_sync(FULL, steps, o);
    }
    if ((threadIdx.x & 31) == 0) { s_tmp[threadIdx.x >> 5] = P; s_tmp[16 + (threadIdx.x >> 5)] = steps; }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long tp = 0, ts = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { tp += s_tmp[w]; ts += s_tmp[16 + w]; }
        I->n_steps = ts;
        I->n_members = ts;
        if (s_bad) { I->status = RR_ERR_ARG; }
        else if (k > 0x3fffffff || tp > 0x7fffffffLL) { I->status = RR_ERR_ARG; }
        else if (ts > I->cap_members || (ts > 0 && (!I->members || !I->ops))) {
            I->status = RR_ERR_CAPACITY;
            I->n_ops = ts;                      // upper bound
        } else {
            bool ok = true;
            const unsigned long long cells = (unsigned long long)m * n;
            ws.P = tp;
            ws.pairOff = (int32_t *)arena_alloc(A, 4ull * (k + 1), &ok);
            ws.nextAt = (int32_t *)arena_alloc(A, 4ull * (tp + 1), &ok);
            ws.colOff = (int32_t *)arena_alloc(A, 4ull * (n + 1), &ok);
            ws.colCur = (int32_t *)arena_alloc(A, 4ull * (n + 1), &ok);
            ws.colList = (int32_t *)arena_alloc(A, 4ull * (k + 1), &ok);
            ws.rowOff = (int32_t *)arena_alloc(A, 4ull * (m + 1), &ok);
            ws.rowCur = (int32_t *)arena_alloc(A, 4ull * (m + 1), &ok);
            ws.rowList = (int32_t *)arena_alloc(A, 4ull * (k + 1), &ok);
            ws.firstH = (int32_t *)arena_alloc(A, 4ull * cells, &ok);
            ws.succCnt = (int32_t *)arena_alloc(A, 4ull * (k + 1), &ok);
            ws.indeg = (int32_t *)arena_alloc(A, 4ull * (k + 1), &ok);
            ws.rec = (int4 *)arena_alloc(A, 32ull * (k + 1), &ok);   // record, successors: one 32 B sector
            ws.succ4 = ws.rec + 1;
            ws.ready0 = (int32_t *)arena_alloc(A, 4ull * (k + 1) + 16, &ok);
            ws.slotOvf = arena_alloc(A, 40ull * (k + 1), &ok);
            ws.ovfFree = (int32_t *)arena_alloc(A, 4ull * (k + 1), &ok);
            // a path has at most as many distinct successors as vertices: they
            // are stored at the path's vertex offset, so no count pass or scan
            ws.succ = (int32_t *)arena_alloc(A, 4ull * (tp + 1), &ok);
            ws.lbStatus = nullptr;
            ws.lbCounter = nullptr;
            if (!ok) I->status = RR_ERR_WORKSPACE;
        }
    }
    __syncthreads();
    if (!live(I)) return;
    // pairOff = exclusive scan of (len + 1); zero the counters
    for (int64_t b = threadIdx.x; b < k; b += blockDim.x) {
        const rr_move p = I->moves[b];
        ws.pairOff[b] = iabs(p.dst_col - p.src_col) + iabs(p.dst_row - p.src_row) + 1;
        ws.indeg[b] = 0;
    }
    if (threadIdx.x == 0) ws.ready0[k] = 0;      // count of initially ready moves
    for (int c = threadIdx.x; c <= n; c += blockDim.x) { ws.colOff[c] = 0; ws.colCur[c] = 0; }
    for (int r = threadIdx.x; r <= m; r += blockDim.x) { ws.rowOff[r] = 0; ws.rowCur[r] = 0; }
    __syncthreads();
    const long long tot = block_exclusive_scan(ws.pairOff, (int)k, s_tmp);
    if (threadIdx.x == 0) ws.pairOff[k] = (int32_t)tot;
}

// Path-vertex offsets of a large move list: pairOff[b] = sum over a < b of
// (path length + 1), by a single pass of decoupled look-back (Merrill and
// Garland, "Single-pass parallel prefix scan with decoupled look-back",
// 2016). Blocks take tiles of LB_TILE moves in order from the instance's
// counter (so every tile a block waits on is held by a running block); a
// tile publishes its aggregate at once and, once its exclusive prefix is
// known from the preceding tiles' words, its inclusive prefix. Status word:
// flag in the top two bits (0 not ready, 1 aggregate, 2 inclusive prefix),
// value in the low 62. Waits are bounded: a block that sees no progress for
// LB_SPIN_LIMIT polls sets RR_ERR_TIMEOUT and stops. The same pass checks
// every move, clears the in-degrees, and the block of the last tile, which
// learns the total, counts the elementary steps, checks the output room and
// allocates the vertex-sized arrays.
constexpr unsigned long long LB_AGG = 1ull << 62, LB_INCL = 2ull << 62, LB_VAL = (1ull << 62) - 1;
constexpr int LB_SPIN_LIMIT = 1 << 22;

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ inline void s_pairoff_lookback(const Blk B, rr_instance *inst, JobWS *wsv, int count, Arena A)
{
    __shared__ long long s_warp[LB_THREADS / 32];
    __shared__ long long s_excl;
    __shared__ int s_tile, s_stop;
    const int q = B.y;
    if (q >= count) return;
    rr_instance *I = &inst[q];
    if (!live(I)) return;
    JobWS &ws = wsv[q];
    if (!ws.lbStatus) return;
    const int64_t k = I->n_moves;
    const int ntile = (int)((k + LB_TILE - 1) / LB_TILE);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (;;) {
        if (tid == 0) { s_tile = atomicAdd(ws.lbCounter, 1); s_stop = 0; }
        __syncthreads();
        const int tile = s_tile;
        if (tile >= ntile) break;
        // this thread's LB_ITEMS consecutive moves
        const int64_t b0 = (int64_t)tile * LB_TILE + (int64_t)tid * LB_ITEMS;
        int v[LB_ITEMS];
        long long sum = 0;
        bool bad = false;
        const int m = I->m, n = I->n;
#pragma unroll
        for (int u = 0; u < LB_ITEMS; ++u) {
            const int64_t b = b0 + u;
            v[u] = 0;
            if (b < k) {
                const rr_move p = I->moves[b];
                bad |= p.src_row < 0 || p.src_row >= m || p.dst_row < 0 || p.dst_row >= m || p.src_col < 0 ||
                       p.src_col >= n || p.dst_col < 0 || p.dst_col >= n ||
                       (p.src_row == p.dst_row && p.src_col == p.dst_col);
                v[u] = iabs(p.dst_col - p.src_col) + iabs(p.dst_row - p.src_row) + 1;
                ws.indeg[b] = 0;
            }
            sum += v[u];
        }
        if (bad) set_status(I, RR_ERR_ARG);
        // block scan of the thread sums
        long long incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long t = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) s_warp[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            const long long w = lane < LB_THREADS / 32 ? s_warp[lane] : 0;
            long long wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long t = __shfl_up_sync(FULL, wi, o);
                if (lane >= o) wi += t;
            }
            if (lane < LB_THREADS / 32) s_warp[lane] = wi - w;
            const long long agg = __shfl_sync(FULL, wi, 31);
            if (lane == 0) {
                unsigned long long *st = ws.lbStatus;
                long long excl = 0;
                if (tile == 0) {
                    st_release_u64(&st[0], LB_INCL | (unsigned long long)agg);
                } else {
                    st_release_u64(&st[tile], LB_AGG | (unsigned long long)agg);
                    int j = tile - 1, spins = 0;
                    while (j >= 0) {
                        const unsigned long long w2 = ld_acquire_u64(&st[j]);
                        const unsigned long long f = w2 & ~LB_VAL;
                        if (f == 0ull) {
                            if (++spins > LB_SPIN_LIMIT) { s_stop = 1; break; }
                            __nanosleep(32);
                            continue;
                        }
                        spins = 0;
                        excl += (long long)(w2 & LB_VAL);
                        if (f == LB_INCL) break;
                        --j;
                    }
                    if (!s_stop) st_release_u64(&st[tile], LB_INCL | (unsigned long long)(excl + agg));
                }
                s_excl = excl;
                if (tile == ntile - 1 && !s_stop) {
                    // the total: elementary steps, the room they need, and
                    // the vertex-sized arrays (as the one-block set-up does)
                    const long long tp = excl + agg, ts = tp - k;
                    I->n_steps = ts;
                    I->n_members = ts;
                    if (tp > 0x7fffffffLL) {
                        set_status(I, RR_ERR_ARG);
                    } else if (ts > I->cap_members || (ts > 0 && (!I->members || !I->ops))) {
                        if (atomicCAS(&I->status, RR_OK, RR_ERR_CAPACITY) == RR_OK) I->n_ops = ts;
                    } else {
                        bool ok = true;
                        ws.P = tp;
                        ws.pairOff[k] = (int32_t)tp;
                        ws.nextAt = (int32_t *)arena_alloc(A, 4ull * (tp + 1), &ok);
                        ws.succ = (int32_t *)arena_alloc(A, 4ull * (tp + 1), &ok);
                        if (!ok) set_status(I, RR_ERR_WORKSPACE);
                    }
                }
            }
        }
        __syncthreads();
        if (s_stop) {
            if (tid == 0) set_status(I, RR_ERR_TIMEOUT);
            break;
        }
        long long run = s_excl + s_warp[wid] + incl - sum;
#pragma unroll
        for (int u = 0; u < LB_ITEMS; ++u) {
            const int64_t b = b0 + u;
            if (b < k) ws.pairOff[b] = (int32_t)run;
            run += v[u];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- Gamma
// Vertex (r, c) is covered by the vertical parts of the moves ending in
// column c (the corner of an L-move included) and by the horizontal parts of
// the L-moves running along row r (their destination column excluded). Two
// sweeps in id order -- one per row over the L-moves on it, one per column
// over the moves ending there -- give each vertex's horizontal and vertical
// coverers as two id-ordered chains. In red-rec plans every vertical
// coverer precedes every horizontal one (a corridor only crosses a column
// after that column's moves were emitted), so the chains are concatenated;
// elsewhere (bird's corridors cross columns solved later) the column sweep
// merges the two chains of that vertex by id (a chain holds each move at
// most once, so a merge takes at most k steps; more is an invariant failure).

__device__ inline void s_gcount(const Blk B, rr_instance *inst, JobWS *wsv, int count)
{
    const int q = B.y;
    if (q >= count) return;
    const rr_instance *I = &inst[q];
    if (!live(I)) return;
    JobWS &ws = wsv[q];
    const int64_t k = I->n_moves;
    for (int64_t b = B.x * blockDim.x + threadIdx.x; b < k; b += (int64_t)B.gx * blockDim.x) {
        const rr_move p = I->moves[b];
        atomicAdd(&ws.colCur[p.dst_col], 1);
        if (p.src_col != p.dst_col) atomicAdd(&ws.rowCur[p.src_row], 1);
    }
}

__device__ inline void s_gscan(const Blk B, rr_instance *inst, JobWS *wsv, int count)
{
    const int q = B.x;
    if (q >= count) return;
    const rr_instance *I = &inst[q];
    if (!live(I)) return;
    JobWS &ws = wsv[q];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (wid > 1) return;
    // warp 0: columns, warp 1: rows
    const int len = wid == 0 ? I->n : I->m;
    int32_t *cnt = wid == 0 ? ws.colCur : ws.rowCur, *off = wid == 0 ? ws.colOff : ws.rowOff;
    int carry = 0;
    for (int base = 0; base < len; base += 32) {
        const int i = base + lane;
        const int v = i < len ? cnt[i] : 0;
        const int incl = warp_incl_scan(v);
        if (i < len) { off[i] = carry + incl - v; cnt[i] = carry + incl - v; }
        carry += __shfl_sync(FULL, incl, 31);
    }
    if (lane == 0) off[len] = carry;
}

__device__ inline void s_gfill(const Blk B, rr_instance *inst, JobWS *wsv, int count)
{
    const int q = B.y;
    if (q >= count) return;
    const rr_instance *I = &inst[q];
    if (!live(I)) return;
    JobWS &ws = wsv[q];
    const int64_t k = I->n_moves;
    for (int64_t b = B.x * blockDim.x + threadIdx.x; b < k; b += (int64_t)B.gx * blockDim.x) {
        const rr_move p = I->moves[b];
        ws.colList[atomicAdd(&ws.colCur[p.dst_col], 1)] = (int32_t)b;
        if (p.src_col != p.dst_col) ws.rowList[atomicAdd(&ws.rowCur[p.src_row], 1)] = (int32_t)b;
    }
}

// Sort a[0..n) of int32 ascending with one warp (registers up to 32, else a
// shared-memory bitonic network over buf, sized for the next power of two).
__device__ inline void warp_sort32(int32_t *a, int n, int32_t *buf)
{
    const int lane = threadIdx.x & 31;
    if (n <= 1) return;
    if (n <= 32) {
        int v = lane < n ? a[lane] : 0x7fffffff;
#pragma unroll
        for (int kk = 2; kk <= 32; kk <<= 1) {
#pragma unroll
            for (int jj = kk >> 1; jj > 0; jj >>= 1) {
                const int o = __shfl_xor_sync(FULL, v, jj);
                const bool up = (lane & kk) == 0, low = (lane & jj) == 0;
                v = (low == up) ? min(v, o) : max(v, o);
            }
        }
        if (lane < n) a[lane] = v;
        __syncwarp();
        return;
    }
    int P = 1;
    while (P < n) P <<= 1;
    for (int i = lane; i < P; i += 32) buf[i] = i < n ? a[i] : 0x7fffffff;
    __syncwarp();
    for (int k = 2; k <= P; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = lane; i < P; i += 32) {
                const int ij = i ^ j;
                if (ij > i) {
                    const int x = buf[i], y = buf[ij];
                    if ((x > y) == ((i & k) == 0)) { buf[i] = y; buf[ij] = x; }
                }
            }
            __syncwarp();
        }
    for (int i = lane; i < n; i += 32) a[i] = buf[i];
    __syncwarp();
}

// Order every column list and row list by id (one warp per list). Lists of
// red-rec plans are mostly ascending already.
__device__ inline void s_gsort(const Blk B, rr_instance *inst, JobWS *wsv, int count, int bufLen)
{
    extern __shared__ int32_t sortbuf[];
    const int q = B.y;
    if (q >= count) return;
    const rr_instance *I = &inst[q];
    if (!live(I)) return;
    JobWS &ws = wsv[q];
    const int lane = threadIdx.x & 31;
    int32_t *buf = sortbuf + (threadIdx.x >> 5) * bufLen;
    const int nl = I->n + I->m;
    for (int l = B.x * (blockDim.x >> 5) + (threadIdx.x >> 5); l < nl; l += B.gx * (blockDim.x >> 5)) {
        const bool col = l < I->n;
        const int idx = col ? l : l - I->n;
        int32_t *a = col ? ws.colList + ws.colOff[idx] : ws.rowList + ws.rowOff[idx];
        const int len = col ? ws.colOff[idx + 1] - ws.colOff[idx] : ws.rowOff[idx + 1] - ws.rowOff[idx];
        bool sorted = true;
        for (int i = lane; i + 1 < len; i += 32) sorted &= a[i] < a[i + 1];
        if (__all_sync(FULL, sorted)) continue;
        warp_sort32(a, len, buf);
    }
}

// Row sweep: the L-moves along each row in id order; each vertex's
// consecutive horizontal coverers are linked, the first is recorded.
__device__ inline void s_gsweep_h(const Blk B, rr_instance *inst, JobWS *wsv, int count, int lineCap)
{
    extern __shared__ int32_t sweepbuf[];
    const int q = B.y;
    if (q >= count) return;
    const rr_instance *I = &inst[q];
    if (!live(I)) return;
    JobWS &ws = wsv[q];
    const int lane = threadIdx.x & 31;
    const int n = I->n, m = I->m;
    int32_t *lastPos = sweepbuf + (threadIdx.x >> 5) * lineCap;
    for (int r = B.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < m; r += B.gx * (blockDim.x >> 5)) {
        for (int c = lane; c < n; c += 32) { lastPos[c] = -1; ws.firstH[(size_t)r * n + c] = -1; }
        __syncwarp();
        for (int e = ws.rowOff[r]; e < ws.rowOff[r + 1]; ++e) {
            const int b = ws.rowList[e];
            const rr_move p = I->moves[b];
            const int step = p.dst_col > p.src_col ? 1 : -1;
            const int hl = iabs(p.dst_col - p.src_col);
            const int base = ws.pairOff[b];
            for (int t = lane; t < hl; t += 32) {       // the destination column is the corner
                const int c = p.src_col + t * step;
                const int prev = lastPos[c];
                if (prev >= 0) ws.nextAt[prev] = b;
                else ws.firstH[(size_t)r * n + c] = b;
                lastPos[c] = base + t;
            }
            __syncwarp();
        }
        for (int c = lane; c < n; c += 32)
            if (lastPos[c] >= 0) ws.nextAt[lastPos[c]] = -1;
        __syncwarp();
    }
}


// Column sweep: the moves ending in each column in id order; consecutive
// vertical coverers are linked, the last one to the vertex's first
// horizontal coverer. Where a horizontal coverer precedes a vertical one (a
// bird corridor through a column solved later), the two id-ordered chains of
// that vertex are merged by id instead.
__device__ inline void s_gsweep_v(const Blk B, rr_instance *inst, JobWS *wsv, int count, int lineCap)
{
    extern __shared__ int32_t sweepbuf[];
    const int q = B.y;
    if (q >= count) return;
    rr_instance *I = &inst[q];
    if (!live(I)) return;
    JobWS &ws = wsv[q];
    const int lane = threadIdx.x & 31;
    const int n = I->n, m = I->m;
    const int64_t k = I->n_moves;
    int32_t *lastPos = sweepbuf + (threadIdx.x >> 5) * 3 * lineCap;
    int32_t *lastId = lastPos + lineCap;
    int32_t *firstId = lastId + lineCap;
    for (int c = B.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < n; c += B.gx * (blockDim.x >> 5)) {
        for (int r = lane; r < m; r += 32) lastPos[r] = -1;
        __syncwarp();
        for (int e = ws.colOff[c]; e < ws.colOff[c + 1]; ++e) {
            const int b = ws.colList[e];
            const rr_move p = I->moves[b];
            const int step = p.dst_row > p.src_row ? 1 : -1;
            const int hl = iabs(p.dst_col - p.src_col), vl = iabs(p.dst_row - p.src_row);
            const int base = ws.pairOff[b] + hl;
            for (int t = lane; t <= vl; t += 32) {      // t = 0 is the corner / the source
                const int r = p.src_row + t * step;
                const int prev = lastPos[r];
                if (prev >= 0) ws.nextAt[prev] = b;
                else firstId[r] = b;
                lastPos[r] = base + t;
                lastId[r] = b;
            }
            __syncwarp();
        }
        bool bad = false;
        for (int r = lane; r < m; r += 32) {
            if (lastPos[r] < 0) continue;
            const int f = ws.firstH[(size_t)r * n + c];
            if (f < 0 || f > lastId[r]) {              // every vertical coverer first
                ws.nextAt[lastPos[r]] = f;
                continue;
            }
            // merge: take the smaller id of the two chain heads, link it
            // after the previous one, advance its chain
            int v = firstId[r], h = f, prevEntry = -1;
            int64_t steps = 0;
            for (; (v >= 0 || h >= 0) && steps <= k; ++steps) {   // a chain holds each move at most once
                const bool takeV = h < 0 || (v >= 0 && v < h);
                const int x = takeV ? v : h;
                const rr_move p = I->moves[x];
                const int e = ws.pairOff[x] + (takeV ? iabs(p.dst_col - p.src_col) + iabs(r - p.src_row)
                                                     : iabs(c - p.src_col));
                const int nx = (takeV && e == lastPos[r]) ? -1 : ws.nextAt[e];
                if (prevEntry >= 0) ws.nextAt[prevEntry] = x;
                prevEntry = e;
                if (takeV) v = nx; else h = nx;
            }
            if (prevEntry >= 0) ws.nextAt[prevEntry] = -1;
            bad |= steps > k;
        }
        if (__any_sync(FULL, bad) && lane == 0) set_status(I, RR_ERR_INTERNAL);
        __syncwarp();
    }
}

// Distinct successors of one path, in first-occurrence order, written to
// out[0..) (each also counted in the successor's in-degree); returns their
// number. Consecutive path vertices mostly share their next path, so most
// entries repeat the previous one; a new value is checked against the first
// four successors (registers) and then against the rest already written
// (read back from out, which only this thread writes). The path's entries
// are read 16 bytes at a time once aligned.
__device__ inline int distinct_succ(const int32_t *seq, int len, int32_t *out, int32_t *indeg)
{
    int cnt = 0;
    int32_t last = -1, b0 = -1, b1 = -1, b2 = -1, b3 = -1;
    auto visit = [&](int32_t v) {
        if (v < 0 || v == last) return;
        last = v;
        if (v == b0 || v == b1 || v == b2 || v == b3) return;
        for (int u = 4; u < cnt; ++u)
            if (out[u] == v) return;
        if (cnt == 0) b0 = v; else if (cnt == 1) b1 = v; else if (cnt == 2) b2 = v; else if (cnt == 3) b3 = v;
        out[cnt++] = v;
        atomicAdd(&indeg[v], 1);
    };
    int t = 0;
    const int head = min(len, (int)((4u - (unsigned)(((uintptr_t)seq >> 2) & 3u)) & 3u));
    for (; t < head; ++t) visit(seq[t]);
    for (; t + 4 <= len; t += 4) {
        const int4 q = *reinterpret_cast<const int4 *>(seq + t);
        visit(q.x); visit(q.y); visit(q.z); visit(q.w);
    }
    for (; t < len; ++t) visit(seq[t]);
    return cnt;
}

// Distinct successors of every path, written at the path's vertex offset,
// their count, and the in-degree of every successor.
__device__ inline void s_bsucc(const Blk B, rr_instance *inst, JobWS *wsv, int count)
{
    const int q = B.y;
    if (q >= count) return;
    const rr_instance *I = &inst[q];
    if (!live(I)) return;
    JobWS &ws = wsv[q];
    const int64_t k = I->n_moves;
    for (int64_t b = B.x * blockDim.x + threadIdx.x; b < k; b += (int64_t)B.gx * blockDim.x) {
        const int lo = ws.pairOff[b], hi = ws.pairOff[b + 1];
        ws.succCnt[b] = distinct_succ(ws.nextAt + lo, hi - lo, ws.succ + lo, ws.indeg);
    }
}

// Per-move records for the simulation: packed geometry, successor count and
// the first four successors (flagged when the successor has no other
// predecessor); later successors are flagged in place. Moves without
// predecessors are listed as initially ready.
__device__ inline void s_brec(const Blk B, rr_instance *inst, JobWS *wsv, int count)
{
    const int q = B.y;
    if (q >= count) return;
    const rr_instance *I = &inst[q];
    if (!live(I)) return;
    JobWS &ws = wsv[q];
    const int64_t k = I->n_moves;
    for (int64_t b = B.x * blockDim.x + threadIdx.x; b < k; b += (int64_t)B.gx * blockDim.x) {
        const rr_move p = I->moves[b];
        const int lo = ws.pairOff[b], hi = lo + ws.succCnt[b];
        int4 r;
        r.x = (p.src_row & 0xffff) | (p.src_col << 16);
        r.y = (p.dst_row & 0xffff) | (p.dst_col << 16);
        r.z = hi - lo;
        r.w = lo + 4;
        int v[4] = {-1, -1, -1, -1};
        for (int e = lo; e < hi; ++e) {
            const int32_t sId = ws.succ[e];
            const int32_t f = sId | (ws.indeg[sId] == 1 ? SUCC_SINGLE : 0);
            if (e - lo < 4) v[e - lo] = f; else ws.succ[e] = f;
        }
        ws.rec[2 * b] = r;
        ws.rec[2 * b + 1] = make_int4(v[0], v[1], v[2], v[3]);
        if (ws.indeg[b] == 0) ws.ready0[atomicAdd(&ws.ready0[k], 1)] = (int32_t)b;
    }
}

// ---------------------------------------------------------- simulation
//
// The ready moves other than the leader live in a slot table (structure of
// arrays; shared memory up to its capacity, then a global overflow area with
// the same layout); the leader is held in registers (LeaderState).
// The moves of the current batch other than the leader ("members") are kept
// in a persistent array sorted by id; every other ready move ("static") is
// linked into two lists, one per (direction, row) and one per (direction,
// column), and flagged in per-direction bitmaps of non-empty rows (vertical
// directions) or columns (horizontal ones) for pickup detection.
//
// Members always share one line (a row or a column) and one direction. At a
// segment boundary the candidates of the leader's row are the statics of that
// row list plus the members if they form that row (likewise for its column);
// so a segment walks two lists, usually short, and merges the newcomers. The
// batch is dissolved back into the lists only when the leader's line or
// direction no longer matches the members'.

constexpr int KEY_LIVE = 1 << 22;
constexpr int KEY_MEM = 1 << 23;
constexpr int INTMAX = 0x7fffffff;

template <typename IX> struct SlotSoA {
    int32_t *key;     // row | col << 10 | dir << 20 | KEY_LIVE [| KEY_MEM]; 0 when free
    int32_t *id;      // move id, INT_MAX when free
    int16_t *t;       // elementary steps done (paths are shorter than 2 048 steps)
    int16_t *legEnd;  // t at the end of the current straight leg
    int16_t *dstRow;  // destination row: where the last (vertical) leg ends
    IX *rp, *rn, *cp, *cn;        // static-list links (slot indices, -1)
    // a move's successors are read from its record when it finishes: only
    // the leader and the members ever finish
};

// The narrow simulation (WIDE false) keeps every slot in shared memory and
// gives up on an instance that needs more (it is retried by the wide one);
// the wide simulation spills slots beyond the shared capacity C to a global
// overflow area. Peak demand on red-rec plans is two ready moves per column
// (one chain head per vertical direction), within the shared capacity.
template <typename IX, bool WIDE> struct Sim {
    using ix = IX;
    static constexpr bool wide = WIDE;
    SlotSoA<IX> sm, gm;
    int C, m, n, Wm, Wn;
    int16_t *freeStk;
    int32_t *map;
    IX *rowHead, *colHead;          // [4][m], [4][n] static lists
    int32_t *ovfFree;               // recycled overflow slots (global)
    uint32_t *rowBits, *colBits;    // [2][Wm] (dirs 0, 1), [2][Wn] (dirs 2, 3)
    int32_t *Mid, *Msl;             // members sorted by id
    long long *Kb;                  // sort / merge buffer
    int32_t *sbuf;
};

// A slot field: shared memory below the capacity C, the global overflow area
// above it. Loads and stores branch on the index (rather than selecting a
// pointer) so that the common shared-memory case stays a shared access.
template <typename T> struct SlotRef {
    T *s, *g;
    int i, C;
    __device__ __forceinline__ operator T() const { return i < C ? s[i] : g[i - C]; }
    __device__ __forceinline__ SlotRef &operator=(T v)
    {
        if (i < C) s[i] = v; else g[i - C] = v;
        return *this;
    }
};
template <bool WIDE, typename T> struct SlotAt {
    static __device__ __forceinline__ T &at(T *s, T *, int i, int) { return s[i]; }
};
template <typename T> struct SlotAt<true, T> {
    static __device__ __forceinline__ SlotRef<T> at(T *s, T *g, int i, int C) { return SlotRef<T>{s, g, i, C}; }
};
#define SLOTF(X, f, i)                                                                         \
    (SlotAt<std::decay_t<decltype(X)>::wide, std::remove_reference_t<decltype(*(X).sm.f)>>::at( \
        (X).sm.f, (X).gm.f, (int)(i), (X).C))

__device__ __forceinline__ int key_of(int r, int c, int d) { return r | (c << 10) | (d << 20) | KEY_LIVE; }
__device__ __forceinline__ int key_r(int k) { return k & 1023; }
__device__ __forceinline__ int key_c(int k) { return (k >> 10) & 1023; }
__device__ __forceinline__ int key_d(int k) { return (k >> 20) & 3; }

// a % b for 0 <= a <= 32 < 2^24 and b >= 1: a float quotient, corrected
// by one either way (exact: the error of the product is far below 1)
__device__ __forceinline__ int small_mod(int a, int b)
{
    const int q = __float2int_rz((float)a * __frcp_rn((float)b));
    int r = a - q * b;
    if (r < 0) r += b;
    if (r >= b) r -= b;
    return r;
}

template <class S>
__device__ __forceinline__ void bits_set(const S &X, int d, int r, int c)
{
    using IX = typename S::ix;
    if (d < 2) atomicOr(&X.rowBits[d * X.Wm + (r >> 5)], 1u << (r & 31));
    else atomicOr(&X.colBits[(d - 2) * X.Wn + (c >> 5)], 1u << (c & 31));
}

// Static-list maintenance. push/remove touch the row list and the column
// list of the slot's current key; callers that run them on several lanes at
// once must guarantee distinct lists (see dissolve()).
template <class S>
__device__ void push_row(const S &X, int si, int key)
{
    using IX = typename S::ix;
    IX *h = &X.rowHead[key_d(key) * X.m + key_r(key)];
    SLOTF(X, rp, si) = (IX)-1; SLOTF(X, rn, si) = *h;
    if (*h >= 0) SLOTF(X, rp, *h) = (IX)si;
    *h = (IX)si;
    if (key_d(key) < 2) atomicOr(&X.rowBits[key_d(key) * X.Wm + (key_r(key) >> 5)], 1u << (key_r(key) & 31));
}
template <class S>
__device__ void push_col(const S &X, int si, int key)
{
    using IX = typename S::ix;
    IX *h = &X.colHead[key_d(key) * X.n + key_c(key)];
    SLOTF(X, cp, si) = (IX)-1; SLOTF(X, cn, si) = *h;
    if (*h >= 0) SLOTF(X, cp, *h) = (IX)si;
    *h = (IX)si;
    if (key_d(key) >= 2) atomicOr(&X.colBits[(key_d(key) - 2) * X.Wn + (key_c(key) >> 5)], 1u << (key_c(key) & 31));
}
template <class S>
__device__ void unlink_row(const S &X, int si, int key)
{
    using IX = typename S::ix;
    const int p = SLOTF(X, rp, si), q = SLOTF(X, rn, si);
    IX *h = &X.rowHead[key_d(key) * X.m + key_r(key)];
    if (p >= 0) SLOTF(X, rn, p) = (IX)q; else *h = (IX)q;
    if (q >= 0) SLOTF(X, rp, q) = (IX)p;
    if (*h < 0 && key_d(key) < 2) atomicAnd(&X.rowBits[key_d(key) * X.Wm + (key_r(key) >> 5)], ~(1u << (key_r(key) & 31)));
}
template <class S>
__device__ void unlink_col(const S &X, int si, int key)
{
    using IX = typename S::ix;
    const int p = SLOTF(X, cp, si), q = SLOTF(X, cn, si);
    IX *h = &X.colHead[key_d(key) * X.n + key_c(key)];
    if (p >= 0) SLOTF(X, cn, p) = (IX)q; else *h = (IX)q;
    if (q >= 0) SLOTF(X, cp, q) = (IX)p;
    if (*h < 0 && key_d(key) >= 2) atomicAnd(&X.colBits[(key_d(key) - 2) * X.Wn + (key_c(key) >> 5)], ~(1u << (key_c(key) & 31)));
}

// Link a slot into its row list and its column list (both head loads first:
// the two lists are independent).
template <class S>
__device__ __forceinline__ void push_both(const S &X, int si, int key)
{
    using IX = typename S::ix;
    IX *hr = &X.rowHead[key_d(key) * X.m + key_r(key)];
    IX *hc = &X.colHead[key_d(key) * X.n + key_c(key)];
    const int oldR = *hr, oldC = *hc;
    SLOTF(X, rp, si) = (IX)-1; SLOTF(X, rn, si) = (IX)oldR;
    SLOTF(X, cp, si) = (IX)-1; SLOTF(X, cn, si) = (IX)oldC;
    if (oldR >= 0) SLOTF(X, rp, oldR) = (IX)si;
    if (oldC >= 0) SLOTF(X, cp, oldC) = (IX)si;
    *hr = (IX)si;
    *hc = (IX)si;
    if (key_d(key) < 2) atomicOr(&X.rowBits[key_d(key) * X.Wm + (key_r(key) >> 5)], 1u << (key_r(key) & 31));
    else atomicOr(&X.colBits[(key_d(key) - 2) * X.Wn + (key_c(key) >> 5)], 1u << (key_c(key) & 31));
}
// Lanes in `pend` link their slots, one lane at a time (two of them may
// share a list).
template <class S>
__device__ __forceinline__ void push_lanes(const S &X, unsigned pend, int si, int key)
{
    using IX = typename S::ix;
    const int lane = threadIdx.x & 31;
    for (; pend; pend &= pend - 1) {
        if (lane == __ffs(pend) - 1) push_both(X, si, key);
        __syncwarp();
    }
}

// First i in 1..maxq with bit (pos + i*delta) set, or 0 (delta = +-1)
// (warp-uniform arguments; every lane calls it). The bits of the range
// [lo, hi] are read a word per lane, 32 words (1 024 bits) per round, and
// the nearest set bit is found with a ballot and ffs / clz; a range within
// one word needs no vote.
__device__ inline int bit_scan(const uint32_t *b, int limit, int pos, int delta, int maxq)
{
    const int lane = threadIdx.x & 31;
    const int lo = delta > 0 ? pos + 1 : max(0, pos - maxq);
    const int hi = delta > 0 ? min(limit - 1, pos + maxq) : pos - 1;
    if (lo > hi) return 0;
    const int w0 = lo >> 5, w1 = hi >> 5;
    auto masked = [&](int w) {
        uint32_t v = b[w];
        if (w == w0) v &= ~0u << (lo & 31);
        if (w == w1) v &= 0xffffffffu >> (31 - (hi & 31));
        return v;
    };
    if (w0 == w1) {
        const uint32_t v = masked(w0);
        if (!v) return 0;
        const int y = delta > 0 ? (w0 << 5) + __ffs(v) - 1 : (w0 << 5) + 31 - __clz(v);
        return delta > 0 ? y - pos : pos - y;
    }
    const int nw = w1 - w0 + 1;
    for (int r = 0; r < nw; r += 32) {
        // rounds run outward from pos: ascending words when delta > 0
        const int idx = r + lane;
        const int w = delta > 0 ? w0 + idx : w1 - idx;
        const uint32_t v = idx < nw ? masked(w) : 0u;
        const unsigned bal = __ballot_sync(FULL, v != 0u);
        if (bal) {
            const int src = __ffs(bal) - 1;   // the word nearest pos
            const uint32_t vv = __shfl_sync(FULL, v, src);
            const int ws = delta > 0 ? w0 + r + src : w1 - r - src;
            const int y = delta > 0 ? (ws << 5) + __ffs(vv) - 1 : (ws << 5) + 31 - __clz(vv);
            return delta > 0 ? y - pos : pos - y;
        }
    }
    return 0;
}

// Lowest move id held in slots [0, hi) and its slot (warp-cooperative).
template <class S>
__device__ int lowest_slot(const S &X, int hi)
{
    using IX = typename S::ix;
    const int lane = threadIdx.x & 31;
    int best = INTMAX, bs = -1;
    for (int i = lane; i < hi; i += 32) {
        const int id = SLOTF(X, id, i);
        if (id < best) { best = id; bs = i; }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const int ob = __shfl_xor_sync(FULL, best, o), os = __shfl_xor_sync(FULL, bs, o);
        if (ob < best || (ob == best && os < bs)) { best = ob; bs = os; }
    }
    return best == INTMAX ? -1 : bs;
}

// Sort a[0..n) ascending: registers for n <= 32, else a shared-memory
// bitonic network (a must have room for the next power of two).
__device__ inline void warp_sort64(long long *a, int n)
{
    const int lane = threadIdx.x & 31;
    if (n <= 1) return;
    if (n <= 32) {
        long long v = lane < n ? a[lane] : 0x7fffffffffffffffll;
#pragma unroll
        for (int kk = 2; kk <= 32; kk <<= 1) {
#pragma unroll
            for (int jj = kk >> 1; jj > 0; jj >>= 1) {
                const long long o = __shfl_xor_sync(FULL, v, jj);
                const bool up = (lane & kk) == 0, low = (lane & jj) == 0;
                v = (low == up) ? (v < o ? v : o) : (v > o ? v : o);
            }
        }
        if (lane < n) a[lane] = v;
        __syncwarp();
        return;
    }
    int P = 1;
    while (P < n) P <<= 1;
    for (int i = n + lane; i < P; i += 32) a[i] = 0x7fffffffffffffffll;
    __syncwarp();
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = lane; i < P; i += 32) {
                const int ij = i ^ j;
                if (ij > i) {
                    const long long x = a[i], y = a[ij];
                    const bool up = (i & k) == 0;
                    if ((x > y) == up) { a[i] = y; a[ij] = x; }
                }
            }
            __syncwarp();
        }
    }
}

// Allocate `cnt` slots (warp-cooperative); lane `rank` < cnt gets a slot.
// freeTop / ovfUsed / hi are warp-uniform.
template <class S>
__device__ __forceinline__ int alloc_slot(const S &X, int rank, int cnt, int &freeTop, int &ovfFreeTop,
                                          int &ovfUsed, int &hi, int kmax, int *err)
{
    using IX = typename S::ix;
    int si = -1;
    const int fromStack = min(cnt, freeTop);
    const int fromOvf = min(cnt - fromStack, ovfFreeTop);
    if (rank < fromStack) si = X.freeStk[freeTop - 1 - rank];
    else if (rank < fromStack + fromOvf) si = X.ovfFree[ovfFreeTop - 1 - (rank - fromStack)];
    else if (rank < cnt) si = X.C + ovfUsed + (rank - fromStack - fromOvf);
    freeTop -= fromStack;
    ovfFreeTop -= fromOvf;
    ovfUsed += cnt - fromStack - fromOvf;
    // the overflow area holds kmax + 1 slots, and slot indices must stay
    // representable in the link type: beyond either, no slot (nothing is
    // written) and the run ends with an error
    // (narrow: the shared capacity; beyond it the instance is handed to the
    // wide simulation)
    const int lastOk = S::wide ? min(X.C + kmax, sizeof(IX) == 2 ? 32767 : 0x7fffffff) : X.C - 1;
    if (si > lastOk) si = -1;
    if (ovfUsed > kmax || X.C + ovfUsed > lastOk + 1) *err = S::wide ? RR_ERR_INTERNAL : RR_SIM_RETRY;
    hi = S::wide ? X.C + ovfUsed : X.C;   // every slot ever used lies below
    return si;
}

// A newly ready move: fill its slot (the caller links it into the lists).
template <class S>
__device__ __forceinline__ int fill_slot(const S &X, int si, int id, int4 r)
{
    using IX = typename S::ix;
    // the first leg: along the source row if the move changes column, else
    // along the column (an L-path runs row first, then column)
    const int sr = r.x & 0xffff, sc = r.x >> 16, dr = r.y & 0xffff, dc = r.y >> 16;
    const int d = dc != sc ? (dc > sc ? 3 : 2) : (dr > sr ? 1 : 0);
    const int key = key_of(sr, sc, d);
    SLOTF(X, key, si) = key;
    SLOTF(X, id, si) = id;
    SLOTF(X, t, si) = 0;
    SLOTF(X, legEnd, si) = (int16_t)(dc != sc ? iabs(dc - sc) : iabs(dr - sr));
    SLOTF(X, dstRow, si) = (int16_t)dr;
    X.map[id & (MAPN - 1)] = si;
    return key;
}

// Pull a move's own record toward L1: it is read when the move finishes.
__device__ __forceinline__ void prefetch_rec(const JobWS &ws, int id)
{
    asm volatile("prefetch.global.L1 [%0];" ::"l"(ws.rec + 2 * id));
}

// Pull the records of a move's first successors toward L1: they are read when
// the move finishes, a few batches later.
__device__ __forceinline__ void prefetch_succ(const JobWS &ws, int4 s4, int nsucc)
{
    const int v[4] = {s4.x, s4.y, s4.z, s4.w};
#pragma unroll
    for (int e = 0; e < 4; ++e)
        if (e < nsucc) {
            const int4 *a = ws.rec + 2 * (v[e] & SUCC_ID);
            asm volatile("prefetch.global.L1 [%0];" ::"l"(a));
        }
}

// Turn the members back into statics (warp-cooperative). Members share one
// line, so their perpendicular lists are distinct and are pushed in
// parallel; the shared line list gets the members as one spliced chain.
template <class S>
__device__ void dissolve(const S &X, int nm, bool rowLine)
{
    using IX = typename S::ix;
    const int lane = threadIdx.x & 31;
    if (nm <= 0) return;
    const int k0 = SLOTF(X, key, X.Msl[0]) & ~KEY_MEM;
    IX *lineHead = rowLine ? &X.rowHead[key_d(k0) * X.m + key_r(k0)] : &X.colHead[key_d(k0) * X.n + key_c(k0)];
    const int oldHead = *lineHead;
    __syncwarp();
    for (int u = lane; u < nm; u += 32) {
        const int si = X.Msl[u];
        const int key = SLOTF(X, key, si) & ~KEY_MEM;
        SLOTF(X, key, si) = key;
        const int prv = u == 0 ? -1 : X.Msl[u - 1], nxt = u == nm - 1 ? oldHead : X.Msl[u + 1];
        if (rowLine) { SLOTF(X, rp, si) = (IX)prv; SLOTF(X, rn, si) = (IX)nxt; push_col(X, si, key); }
        else { SLOTF(X, cp, si) = (IX)prv; SLOTF(X, cn, si) = (IX)nxt; push_row(X, si, key); }
    }
    __syncwarp();
    if (lane == 0) {
        if (oldHead >= 0) { if (rowLine) SLOTF(X, rp, oldHead) = (IX)X.Msl[nm - 1]; else SLOTF(X, cp, oldHead) = (IX)X.Msl[nm - 1]; }
        *lineHead = (IX)X.Msl[0];
        bits_set(X, key_d(k0), key_r(k0), key_c(k0));
    }
    __syncwarp();
}

// The leader (the lowest unfinished move, which is always ready) lives in
// warp-uniform registers and holds no slot: its key (position, direction),
// steps done, the end of its current leg, its destination row, and the
// successor part of its record (count, overflow offset, first four), loaded
// when it becomes the leader so that the load has long completed when it
// finishes.
struct LeaderState {
    int key = 0, t = 0, legEnd = 0, dstRow = 0, nsu = 0, ov = 0;
    int4 s4 = {-1, -1, -1, -1};
    bool pref = false;   // its successors' records still to be prefetched
};

// A ready move becomes the leader: its state moves from its slot (already
// out of the lists and the members) into the registers and the slot is freed.
template <class S>
__device__ __forceinline__ void leader_from_slot(const S &X, const JobWS &ws, int si, int &L, LeaderState &Ld,
                                                 int &freeTop, int &ovfFreeTop)
{
    using IX = typename S::ix;
    const int lane = threadIdx.x & 31;
    L = SLOTF(X, id, si);
    Ld.key = SLOTF(X, key, si) & ~KEY_MEM;
    Ld.t = SLOTF(X, t, si);
    Ld.legEnd = SLOTF(X, legEnd, si);
    Ld.dstRow = SLOTF(X, dstRow, si);
    const int4 own = ws.rec[2 * L];
    Ld.s4 = ws.rec[2 * L + 1];
    Ld.nsu = own.z;
    Ld.ov = own.w;
    Ld.pref = true;
    __syncwarp();
    if (lane == 0) {
        if (X.map[L & (MAPN - 1)] == si) X.map[L & (MAPN - 1)] = -1;
        SLOTF(X, key, si) = 0;
        SLOTF(X, id, si) = INTMAX;
        if (si < X.C) X.freeStk[freeTop] = (int16_t)si; else X.ovfFree[ovfFreeTop] = si;
    }
    if (si < X.C) ++freeTop; else ++ovfFreeTop;
    __syncwarp();
}

// A move that became ready just now becomes the leader straight from its
// record (the first leg as fill_slot sets it).
__device__ __forceinline__ void leader_from_rec(const JobWS &ws, int id, int4 r, int &L, LeaderState &Ld)
{
    const int sr = r.x & 0xffff, sc = r.x >> 16, dr = r.y & 0xffff, dc = r.y >> 16;
    const int d = dc != sc ? (dc > sc ? 3 : 2) : (dr > sr ? 1 : 0);
    L = id;
    Ld.key = key_of(sr, sc, d);
    Ld.t = 0;
    Ld.legEnd = dc != sc ? iabs(dc - sc) : iabs(dr - sr);
    Ld.dstRow = dr;
    Ld.nsu = r.z;
    Ld.ov = r.w;
    Ld.s4 = ws.rec[2 * id + 1];
    Ld.pref = true;
}

// One round of successor entries, at most one per lane (warp-cooperative):
// e is a flagged successor id, or ~index into the successor array. Each
// entry decrements its move's in-degree (unless the move has no other
// predecessor); moves that become ready take a slot and join the static
// lists, except the move handId (the next leader once the leader has
// finished), whose record is handed back in handRec with hand set.
template <class S>
__device__ __forceinline__ void release_round(const S &X, const JobWS &ws, bool has, int32_t e, int handId,
                                              int &hand, int4 &handRec, int &freeTop, int &ovfFreeTop,
                                              int &ovfUsed, int &hi, int kmax, int *err)
{
    using IX = typename S::ix;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    int ready = -1;
    int4 r = make_int4(0, 0, 0, 0);
    if (has) {
        if (e < 0) e = ws.succ[~e];
        const int id = e & SUCC_ID;
        r = ws.rec[2 * id];   // fetched with the counter update
        if ((e & SUCC_SINGLE) || atomicSub(&ws.indeg[id], 1) == 1) ready = id;
    }
    const unsigned hb = __ballot_sync(FULL, ready >= 0 && ready == handId);
    if (hb) {
        const int src = __ffs(hb) - 1;
        handRec.x = __shfl_sync(FULL, r.x, src);
        handRec.y = __shfl_sync(FULL, r.y, src);
        handRec.z = __shfl_sync(FULL, r.z, src);
        handRec.w = __shfl_sync(FULL, r.w, src);
        hand = 1;
        if (lane == src) ready = -1;
    }
    const unsigned bal = __ballot_sync(FULL, ready >= 0);
    const int cnt = __popc(bal);
    if (cnt) {
        const int si = alloc_slot(X, __popc(bal & lt), cnt, freeTop, ovfFreeTop, ovfUsed, hi, kmax, err);
        int key = 0;
        if (ready >= 0 && si >= 0) key = fill_slot(X, si, ready, r);
        __syncwarp();
        push_lanes(X, __ballot_sync(FULL, ready >= 0 && si >= 0), si, key);
    }
    __syncwarp();
}

// Instance order by side, largest first: a counting sort on max(m, n)
// (one block; positions within a side follow the atomics, which does not
// matter: instances are independent). perm[i] is the instance at position i.
__device__ inline void s_order(const Blk B, const rr_instance *inst, int count, int *perm)
{
    __shared__ int hist[RR_MAX_SIDE + 2];
    for (int i = threadIdx.x; i < RR_MAX_SIDE + 2; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    auto key = [&](int q) { return RR_MAX_SIDE + 1 - min(max(max(inst[q].m, inst[q].n), 0), RR_MAX_SIDE + 1); };
    for (int q = threadIdx.x; q < count; q += blockDim.x) atomicAdd(&hist[key(q)], 1);
    __syncthreads();
    if (threadIdx.x < 32) {              // exclusive scan, one warp
        int carry = 0;
        for (int b = 0; b < RR_MAX_SIDE + 2; b += 32) {
            const int i = b + threadIdx.x;
            const int v = i < RR_MAX_SIDE + 2 ? hist[i] : 0;
            const int inc = warp_incl_scan(v);
            if (i < RR_MAX_SIDE + 2) hist[i] = carry + inc - v;
            carry += __shfl_sync(FULL, inc, 31);
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < count; q += blockDim.x) perm[atomicAdd(&hist[key(q)], 1)] = q;
}

// Descriptor copy in that order (one 128-byte descriptor per block).
__device__ inline void s_gather(const Blk B, const rr_instance *inst, const int *perm, rr_instance *pinst)
{
    const int32_t *src = (const int32_t *)&inst[perm[B.x]];
    int32_t *dst = (int32_t *)&pinst[B.x];
    dst[threadIdx.x] = src[threadIdx.x];
}

// Per-instance outputs back to the caller's descriptors.
__device__ inline void s_scatter(const Blk B, rr_instance *inst, const int *perm, const rr_instance *pinst, int count)
{
    for (int i = B.x * blockDim.x + threadIdx.x; i < count; i += B.gx * blockDim.x) {
        const rr_instance *p = &pinst[i];
        rr_instance *o = &inst[perm[i]];
        o->n_moves = p->n_moves;
        o->n_steps = p->n_steps;
        o->n_ops = p->n_ops;
        o->n_members = p->n_members;
        o->status = p->status;
    }
}

// Instances grouped by size class (largest side <= classSide[c]) so that each
// class's simulation launch gets shared memory sized for its own grids.
__device__ inline void s_classify(const Blk B, rr_instance *inst, int count, int nclass, int max_side, int *classCount,
                           int *classList)
{
    for (int q = B.x * blockDim.x + threadIdx.x; q < count; q += B.gx * blockDim.x) {
        const rr_instance *I = &inst[q];
        if (!live(I)) continue;
        const int side = max(I->m, I->n);
        int c = 0;
        while (c < nclass - 1 && side > class_side(max_side, c, nclass)) ++c;
        classList[c * count + atomicAdd(&classCount[c], 1)] = q;
    }
}

template <typename IX, bool WIDE>
__device__ __forceinline__ void sim_body(const Blk B, rr_instance *inst, JobWS *wsv, int count, const int *classList,
                                         const int *classCount, int slotCap, int lineCap)
{
    extern __shared__ int4 smem_i4[];
    int q = B.x;                  // without a class list: every instance
    if (classList) {
        if ((int)B.x >= *classCount) return;
        q = classList[B.x];
    }
    if (q >= count) return;
    rr_instance *I = &inst[q];
    if (WIDE ? I->status != RR_SIM_RETRY : !live(I)) return;
    JobWS &ws = wsv[q];
    const int k = (int)I->n_moves;
    const int m = I->m, n = I->n;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    if (k == 0) { if (lane == 0) { I->n_ops = 0; I->n_members = 0; } return; }
    if (WIDE) {
        // the narrow pass consumed in-degrees before giving up: recount them
        // from the successor lists, then start over
        for (int b = lane; b < k; b += 32) ws.indeg[b] = 0;
        __syncwarp();
        for (int b = lane; b < k; b += 32) {
            const int lo = ws.pairOff[b], cnt = ws.succCnt[b];
            for (int e = 0; e < cnt; ++e) atomicAdd(&ws.indeg[ws.succ[lo + e] & SUCC_ID], 1);
        }
        __syncwarp();
        __threadfence_block();
        if (lane == 0) I->status = RR_OK;
    }

    // shared-memory layout (mirrored by the launcher's size computation)
    Sim<IX, WIDE> X;
    X.C = slotCap; X.m = m; X.n = n; X.Wm = (m + 31) >> 5; X.Wn = (n + 31) >> 5;
    const int lbuf = 2 * (lineCap + 2);
    X.Kb = (long long *)smem_i4;
    int32_t *p32 = (int32_t *)(X.Kb + lbuf);
    X.sm.key = p32; p32 += slotCap;
    X.sm.id = p32; p32 += slotCap;
    X.map = p32; p32 += MAPN;
    X.Mid = p32; p32 += lineCap + 2;
    X.Msl = p32; p32 += lineCap + 2;
    X.sbuf = p32; p32 += SBUF;
    X.rowBits = (uint32_t *)p32; p32 += 2 * ((lineCap + 31) >> 5);
    X.colBits = (uint32_t *)p32; p32 += 2 * ((lineCap + 31) >> 5);
    IX *pix = (IX *)p32;
    X.sm.rp = pix; pix += slotCap;
    X.sm.rn = pix; pix += slotCap;
    X.sm.cp = pix; pix += slotCap;
    X.sm.cn = pix; pix += slotCap;
    X.rowHead = pix; pix += 4 * lineCap;
    X.colHead = pix; pix += 4 * lineCap;
    int16_t *p16 = (int16_t *)pix;
    X.sm.t = p16; p16 += slotCap;
    X.sm.legEnd = p16; p16 += slotCap;
    X.sm.dstRow = p16; p16 += slotCap;
    X.freeStk = p16;
    X.ovfFree = ws.ovfFree;
    {   // overflow slots (global), same structure
        char *g = (char *)ws.slotOvf;
        const size_t K1 = (size_t)k + 1;
        X.gm.key = (int32_t *)g;           g += 4 * K1;
        X.gm.id = (int32_t *)g;            g += 4 * K1;
        IX **fl[4] = {&X.gm.rp, &X.gm.rn, &X.gm.cp, &X.gm.cn};
        for (int u = 0; u < 4; ++u) { *fl[u] = (IX *)g; g += sizeof(IX) * K1; }
        X.gm.t = (int16_t *)g;             g += 2 * K1;
        X.gm.legEnd = (int16_t *)g;        g += 2 * K1;
        X.gm.dstRow = (int16_t *)g;
    }
    for (int i = lane; i < slotCap; i += 32) { X.sm.key[i] = 0; X.sm.id[i] = INTMAX; X.freeStk[i] = (int16_t)(slotCap - 1 - i); }
    for (int i = lane; i < MAPN; i += 32) X.map[i] = -1;
    for (int i = lane; i < 4 * m; i += 32) X.rowHead[i] = (IX)-1;
    for (int i = lane; i < 4 * n; i += 32) X.colHead[i] = (IX)-1;
    for (int i = lane; i < 2 * X.Wm; i += 32) X.rowBits[i] = 0u;
    for (int i = lane; i < 2 * X.Wn; i += 32) X.colBits[i] = 0u;
    int freeTop = slotCap, ovfFreeTop = 0, ovfUsed = 0, hi = slotCap, err = 0;
    __syncwarp();

    // moves without predecessors become statics
    const int32_t *ready0 = ws.ready0;
    const int nready0 = ready0[k];
    for (int base = 0; base < nready0; base += 32) {
        const int cnt = min(32, nready0 - base);
        int id = -1;
        int4 r = make_int4(0, 0, 0, 0);
        if (lane < cnt) { id = ready0[base + lane]; r = ws.rec[2 * id]; }
        const int si = alloc_slot(X, lane, cnt, freeTop, ovfFreeTop, ovfUsed, hi, k, &err);
        int key = 0;
        if (lane < cnt && si >= 0) key = fill_slot(X, si, id, r);
        __syncwarp();
        push_lanes(X, __ballot_sync(FULL, lane < cnt && si >= 0), si, key);
    }

    const int64_t cap_ops = I->cap_ops, cap_mem = I->cap_members;
    rr_op *ops = I->ops;
    int32_t *mem = I->members;
    int64_t nop = 0, nmem = 0;
    int overflow = 0;
    int Ls = lowest_slot(X, hi);
    int L = Ls >= 0 ? SLOTF(X, id, Ls) : -1;
    // the leader: warp-uniform registers, no slot (see LeaderState)
    LeaderState Ld;
    if (err) {
        // out of slots already (narrow pass): handed to the wide pass
    } else if (L != 0) err = RR_ERR_INTERNAL;
    else {
        if (lane == 0) { const int kk = SLOTF(X, key, Ls); unlink_row(X, Ls, kk); unlink_col(X, Ls, kk); }
        __syncwarp();
        leader_from_slot(X, ws, Ls, L, Ld, freeTop, ovfFreeTop);
    }
    // members: nm of them (leader excluded), on one line of type rowLine at
    // index lineIdx, direction dm
    int nm = 0, dm = -1, lineIdx = -1;
    bool rowLine = true;
    const int64_t guard_max = g_guard_cap > 0 ? g_guard_cap : I->n_steps + 2ll * k + 16;
    int64_t guard = 0;
    // records of up to 32 newcomers: fetched when they join, their
    // successors' records prefetched in the next segment
    int4 nrec = make_int4(0, 0, 0, 0), ns4 = nrec;
    int npref = 0;

    while (!err && L < k) {
        if (++guard > guard_max) { err = RR_ERR_TIMEOUT; break; }
        const int lr = key_r(Ld.key), lc = key_c(Ld.key), d = key_d(Ld.key);
        const int remL = Ld.legEnd - Ld.t;
        const int sgn = (d == 1 || d == 3) ? 1 : -1;
        // members still on the leader's line in the leader's direction?
        if (nm > 0 && !(dm == d && (rowLine ? lineIdx == lr : lineIdx == lc))) { dissolve(X, nm, rowLine); nm = 0; }
        // smallest static id on the leader's row and column (lane 0 walks;
        // nothing to walk when both lists are empty)
        int minA = INTMAX, minB = INTMAX;
        const int hA = X.rowHead[d * m + lr], hB = X.colHead[d * n + lc];
        if (hA >= 0 || hB >= 0) {
            if (lane == 0) {
                int walk = 0;
                for (int p = hA; p >= 0 && walk <= lineCap; p = SLOTF(X, rn, p), ++walk) minA = min(minA, SLOTF(X, id, p));
                for (int p = hB; p >= 0 && walk <= 2 * lineCap; p = SLOTF(X, cn, p), ++walk) minB = min(minB, SLOTF(X, id, p));
                if (walk > 2 * lineCap) err = RR_ERR_INTERNAL;
            }
            minA = __shfl_sync(FULL, minA, 0);
            minB = __shfl_sync(FULL, minB, 0);
            err = __shfl_sync(FULL, err, 0);
            if (err) break;
        }
        if (nm > 0) { if (rowLine) minA = min(minA, X.Mid[0]); else minB = min(minB, X.Mid[0]); }
        // the previous segment's newcomers: their records have arrived,
        // their successors' records are prefetched now
        if (lane < npref) prefetch_succ(ws, ns4, nrec.z);
        npref = 0;
        if (minA != INTMAX || minB != INTMAX) {
            const bool chooseRow = minA < minB;
            if (nm > 0 && chooseRow != rowLine) { dissolve(X, nm, rowLine); nm = 0; }
            // newcomers: every static of the chosen line (the list empties)
            const int h = chooseRow ? X.rowHead[d * m + lr] : X.colHead[d * n + lc];
            int nc = 0;
            if (lane == 0) {
                for (int p = h; p >= 0 && nc <= lineCap; p = chooseRow ? SLOTF(X, rn, p) : SLOTF(X, cn, p))
                    X.Kb[nc++] = ((long long)SLOTF(X, id, p) << 32) | (unsigned)p;
                if (chooseRow) {
                    X.rowHead[d * m + lr] = (IX)-1;
                    if (d < 2) atomicAnd(&X.rowBits[d * X.Wm + (lr >> 5)], ~(1u << (lr & 31)));
                } else {
                    X.colHead[d * n + lc] = (IX)-1;
                    if (d >= 2) atomicAnd(&X.colBits[(d - 2) * X.Wn + (lc >> 5)], ~(1u << (lc & 31)));
                }
            }
            nc = __shfl_sync(FULL, nc, 0);
            if (nm + nc > lineCap) { err = RR_ERR_INTERNAL; break; }
            __syncwarp();
            // unlink each newcomer from its perpendicular list (distinct lists)
            for (int u = lane; u < nc; u += 32) {
                const int si = (int)(X.Kb[u] & 0xffffffff);
                const int key = SLOTF(X, key, si);
                if (chooseRow) unlink_col(X, si, key); else unlink_row(X, si, key);
                SLOTF(X, key, si) = key | KEY_MEM;
                const int id = (int)(X.Kb[u] >> 32);
                if (u < 32) { nrec = ws.rec[2 * id]; ns4 = ws.rec[2 * id + 1]; }
                else prefetch_rec(ws, id);
            }
            __syncwarp();
            // merge the newcomers into the sorted members (keys id << 32 | slot)
            if (nc > 0 && nm <= 32 && nc <= 32) {
                // the usual case, one member and one newcomer per lane: each
                // newcomer's id is broadcast in turn; a member's rank grows by
                // the newcomers below it, a newcomer's rank is the members
                // below it (one vote) plus the newcomers below it (ids are
                // distinct)
                const int mId = lane < nm ? X.Mid[lane] : INTMAX;
                const int mSl = lane < nm ? X.Msl[lane] : 0;
                const long long kn = lane < nc ? X.Kb[lane] : 0ll;
                const int nId = lane < nc ? (int)(kn >> 32) : INTMAX;
                int rM = lane, rN = 0;
                for (int j = 0; j < nc; ++j) {
                    const int o = __shfl_sync(FULL, nId, j);
                    rM += o < mId;
                    rN += o < nId;
                    const int below = __popc(__ballot_sync(FULL, mId < o));
                    if (lane == j) rN += below;
                }
                __syncwarp();
                if (lane < nm) { X.Mid[rM] = mId; X.Msl[rM] = mSl; }
                if (lane < nc) { X.Mid[rN] = nId; X.Msl[rN] = (int)(kn & 0xffffffff); }
                nm += nc;
            } else if (nc > 0) {
                const int tot = nm + nc;
                long long *out = X.Kb + (lineCap + 2);
                if (nc <= 32) {
                    // few newcomers (the usual case): ranks by counting
                    for (int u = lane; u < nm; u += 32) {
                        const long long key = ((long long)X.Mid[u] << 32) | (unsigned)X.Msl[u];
                        int r = 0;
                        for (int j = 0; j < nc; ++j) r += X.Kb[j] < key;
                        out[u + r] = key;
                    }
                    if (lane < nc) {
                        const long long key = X.Kb[lane];
                        int r = 0;
                        for (int j = 0; j < nc; ++j) r += X.Kb[j] < key;
                        int lo = 0, hi2 = nm;
                        while (lo < hi2) {
                            const int md = (lo + hi2) >> 1;
                            if ((((long long)X.Mid[md] << 32) | (unsigned)X.Msl[md]) < key) lo = md + 1; else hi2 = md;
                        }
                        out[r + lo] = key;
                    }
                } else {
                    warp_sort64(X.Kb, nc);
                    for (int u = lane; u < nm; u += 32) {      // member u: rank among newcomers
                        const long long key = ((long long)X.Mid[u] << 32) | (unsigned)X.Msl[u];
                        int lo = 0, hi2 = nc;
                        while (lo < hi2) { const int md = (lo + hi2) >> 1; if (X.Kb[md] < key) lo = md + 1; else hi2 = md; }
                        out[u + lo] = key;
                    }
                    for (int u = lane; u < nc; u += 32) {      // newcomer u: rank among members
                        const long long key = X.Kb[u];
                        int lo = 0, hi2 = nm;
                        while (lo < hi2) {
                            const int md = (lo + hi2) >> 1;
                            if ((((long long)X.Mid[md] << 32) | (unsigned)X.Msl[md]) < key) lo = md + 1; else hi2 = md;
                        }
                        out[u + lo] = key;
                    }
                }
                __syncwarp();
                for (int u = lane; u < tot; u += 32) { X.Mid[u] = (int)(out[u] >> 32); X.Msl[u] = (int)(out[u] & 0xffffffff); }
                nm = tot;
            }
            npref = min(nc, 32);
            rowLine = chooseRow;
            lineIdx = chooseRow ? lr : lc;
            dm = d;
            __syncwarp();
        }
        // segment length: shortest remaining leg, next pickup
        int kseg = remL;
        // up to 32 members: lane u keeps member u's slot, id, key, steps and
        // leg end in registers from here through the advance
        const bool regM = nm > 0 && nm <= 32;
        int mSi = -1, mId = 0, mKey = 0, mT = 0, mLe = 0;
        if (nm > 0) {
            int remM = INTMAX;
            if (regM) {
                if (lane < nm) {
                    mSi = X.Msl[lane];
                    mId = X.Mid[lane];
                    mKey = SLOTF(X, key, mSi);
                    mT = SLOTF(X, t, mSi);
                    mLe = SLOTF(X, legEnd, mSi);
                    remM = mLe - mT;
                }
            } else {
                for (int u = lane; u < nm; u += 32) { const int si = X.Msl[u]; remM = min(remM, SLOTF(X, legEnd, si) - SLOTF(X, t, si)); }
            }
            kseg = min(kseg, __reduce_min_sync(FULL, remM));   // one warp reduction
        }
        if (kseg > 1) {   // a static move of direction d the leader's line reaches
            const int hit = d >= 2 ? bit_scan(X.colBits + (d - 2) * X.Wn, n, lc, sgn, kseg - 1)
                                   : bit_scan(X.rowBits + d * X.Wm, m, lr, sgn, kseg - 1);
            if (hit > 0) kseg = hit;
        }
        if (kseg < 1) { err = RR_ERR_INTERNAL; break; }
        const int ns = nm + 1;

        // kseg identical batches: the leader, then the members in ascending id
        // (a segment holds at most 2 048 batches of at most lineCap + 1 moves,
        // so offsets within it fit 32 bits; the first-member field is the
        // low 32 bits of the member count, as the ABI's int32 field holds it)
        const int addm = kseg * ns;
        if (!overflow && nop + kseg <= cap_ops && nmem + addm <= cap_mem) {
            rr_op *op = ops + nop;
            int32_t *mp = mem + nmem;
            const int32_t f0 = (int32_t)nmem;
            if (ns == 1) {
                for (int i = lane; i < kseg; i += 32) { op[i] = rr_op{d, f0 + i, 1}; mp[i] = L; }
            } else {
                for (int i = lane; i < kseg; i += 32) op[i] = rr_op{d, f0 + i * ns, ns};
                int u = small_mod(lane, ns);
                const int step = small_mod(32, ns);
                for (int i = lane; i < addm; i += 32) {
                    mp[i] = u == 0 ? L : X.Mid[u - 1];
                    u += step;
                    if (u >= ns) u -= ns;
                }
            }
        } else {
            overflow = 1;
        }
        nop += kseg;
        nmem += addm;

        // advance by kseg steps along the current legs (no batch move's leg
        // ends before the segment does); at a leg's end a move finishes on
        // its destination row or turns toward it. The leader first (its
        // registers), then the members: finished members release their
        // successors, members whose leg ended leave the batch and become
        // statics, the others stay members.
        if (Ld.pref) {   // the leader's record has arrived by now
            prefetch_succ(ws, Ld.s4, lane == 0 ? Ld.nsu : 0);
            Ld.pref = false;
        }
        bool lfin = false;
        {
            const int t = Ld.t + kseg;
            const int r_ = lr + (d == 1 ? kseg : d == 0 ? -kseg : 0);
            const int c_ = lc + (d == 3 ? kseg : d == 2 ? -kseg : 0);
            int d_ = d;
            Ld.t = t;
            if (t == Ld.legEnd) {
                if (r_ == Ld.dstRow) lfin = true;
                else { d_ = Ld.dstRow > r_ ? 1 : 0; Ld.legEnd = t + iabs(Ld.dstRow - r_); }
            }
            Ld.key = key_of(r_, c_, d_);
        }
        // once the leader has finished, L + 1 (if it becomes ready now) is the
        // next leader and takes no slot
        const int handId = lfin ? L + 1 : -1;
        int hand = 0;
        int4 handRec = make_int4(0, 0, 0, 0);
        int nkeep = 0;
        for (int u0 = 0; u0 < nm; u0 += 32) {
            const int u = u0 + lane;
            bool fin = false, turn = false;
            const bool act = u < nm;
            int si = -1, nsu = 0, newKey = 0, ov = 0;
            int4 fs4 = make_int4(0, 0, 0, 0);
            if (act) {
                si = regM ? mSi : X.Msl[u];
                const int key = regM ? mKey : SLOTF(X, key, si);
                const int t = (regM ? mT : SLOTF(X, t, si)) + kseg;
                const int le = regM ? mLe : SLOTF(X, legEnd, si);
                int d_ = key_d(key);
                const int r_ = key_r(key) + (d_ == 1 ? kseg : d_ == 0 ? -kseg : 0);
                const int c_ = key_c(key) + (d_ == 3 ? kseg : d_ == 2 ? -kseg : 0);
                int rem = le - t;
                SLOTF(X, t, si) = (int16_t)t;
                if (rem == 0) {
                    const int dr = SLOTF(X, dstRow, si);
                    fin = r_ == dr;
                    d_ = dr > r_ ? 1 : 0;
                    rem = iabs(dr - r_);
                }
                if (fin) {
                    const int id = regM ? mId : SLOTF(X, id, si);
                    const int4 own = ws.rec[2 * id];
                    fs4 = ws.rec[2 * id + 1];
                    nsu = own.z;
                    ov = own.w;
                } else {
                    turn = d_ != d;
                    newKey = key_of(r_, c_, d_) | (turn ? 0 : KEY_MEM);
                    SLOTF(X, key, si) = newKey;
                    if (t + rem != le) SLOTF(X, legEnd, si) = (int16_t)(t + rem);
                }
            }
            // survivors keep their order (stable compaction: straight into the
            // member arrays when they are held in registers, else into Kb)
            const bool keep = act && !fin && !turn;
            const unsigned kb = __ballot_sync(FULL, keep);
            if (regM) {
                __syncwarp();
                if (keep) { X.Mid[__popc(kb & lt)] = mId; X.Msl[__popc(kb & lt)] = si; }
            } else if (keep) {
                X.Kb[nkeep + __popc(kb & lt)] = ((long long)X.Mid[u] << 32) | (unsigned)si;
            }
            nkeep += __popc(kb);
            // members whose leg ended become statics
            push_lanes(X, __ballot_sync(FULL, turn), si, newKey);
            if (!__any_sync(FULL, fin)) continue;     // nothing finished in this chunk
            const int off = warp_incl_scan(nsu) - nsu;
            const int total = __shfl_sync(FULL, off + nsu, 31);
            // free the finished moves' slots first (their successors may take
            // them; shared-memory slots are recycled)
            if (fin) {
                const int id = SLOTF(X, id, si);
                if (X.map[id & (MAPN - 1)] == si) X.map[id & (MAPN - 1)] = -1;
                SLOTF(X, key, si) = 0;
                SLOTF(X, id, si) = INTMAX;
            }
            const bool recyc = fin && si < X.C, recycO = fin && si >= X.C;
            const unsigned fb = __ballot_sync(FULL, recyc), fo = __ballot_sync(FULL, recycO);
            if (recyc) X.freeStk[freeTop + __popc(fb & lt)] = (int16_t)si;
            if (recycO) X.ovfFree[ovfFreeTop + __popc(fo & lt)] = si;
            freeTop += __popc(fb);
            ovfFreeTop += __popc(fo);
            __syncwarp();
            // successor entries of the finished members, in rounds of SBUF
            for (int base = 0; base < total; base += SBUF) {
                if (fin) {
                    for (int e = max(0, base - off); e < nsu && off + e < base + SBUF; ++e)
                        X.sbuf[off + e - base] = e == 0 ? fs4.x : e == 1 ? fs4.y : e == 2 ? fs4.z : e == 3 ? fs4.w
                                                                                                : ~(ov + e - 4);
                }
                __syncwarp();
                const int nb = min(SBUF, total - base);
                for (int b0 = 0; b0 < nb; b0 += 32) {
                    const bool has = b0 + lane < nb;
                    release_round(X, ws, has, has ? X.sbuf[b0 + lane] : 0, handId, hand, handRec, freeTop,
                                  ovfFreeTop, ovfUsed, hi, k, &err);
                }
            }
        }
        // the finished leader's successors, straight from its registers
        if (lfin && Ld.nsu == 1 && (Ld.s4.x & SUCC_SINGLE)) {
            // one successor, with no other predecessor: ready now (uniform)
            const int sid = Ld.s4.x & SUCC_ID;
            const int4 r = ws.rec[2 * sid];
            if (sid == handId) { hand = 1; handRec = r; }
            else {
                const int si = alloc_slot(X, lane, 1, freeTop, ovfFreeTop, ovfUsed, hi, k, &err);
                if (lane == 0 && si >= 0) push_both(X, si, fill_slot(X, si, sid, r));
                __syncwarp();
            }
        } else if (lfin) {
            for (int e0 = 0; e0 < Ld.nsu; e0 += 32) {
                const int e = e0 + lane;
                const int32_t v = e == 0 ? Ld.s4.x : e == 1 ? Ld.s4.y : e == 2 ? Ld.s4.z : e == 3 ? Ld.s4.w
                                                                                            : ~(Ld.ov + e - 4);
                release_round(X, ws, e < Ld.nsu, v, handId, hand, handRec, freeTop, ovfFreeTop, ovfUsed, hi, k,
                              &err);
            }
        }
        if (!regM)
            for (int u = lane; u < nkeep; u += 32) { X.Mid[u] = (int)(X.Kb[u] >> 32); X.Msl[u] = (int)(X.Kb[u] & 0xffffffff); }
        nm = nkeep;
        // a line moving across itself carries its index along
        if (rowLine && d < 2) lineIdx += sgn * kseg;
        if (!rowLine && d >= 2) lineIdx += sgn * kseg;
        __syncwarp();
        if (lfin && !err) {
            // next leader: the lowest unfinished id. L + 1, if it became ready
            // just now, takes over at once; otherwise the lowest id still held
            // (usually L + 1): a member leaves the front of the members, a
            // static its lists
            if (hand) leader_from_rec(ws, L + 1, handRec, L, Ld);
            else {
                int cand = -1;
                const int nx = L + 1;
                if (nx < k) {
                    const int si = X.map[nx & (MAPN - 1)];
                    if (si >= 0 && SLOTF(X, id, si) == nx) cand = si;
                }
                if (cand < 0) cand = lowest_slot(X, hi);
                if (cand < 0) L = k;
                else {
                    const int kk = SLOTF(X, key, cand);
                    if (kk & KEY_MEM) {
                        if (nm == 0 || X.Msl[0] != cand) { err = RR_ERR_INTERNAL; break; }
                        __syncwarp();
                        for (int u = lane; u + 1 < nm; u += 32) X.Kb[u] = ((long long)X.Mid[u + 1] << 32) | (unsigned)X.Msl[u + 1];
                        __syncwarp();
                        --nm;
                        for (int u = lane; u < nm; u += 32) { X.Mid[u] = (int)(X.Kb[u] >> 32); X.Msl[u] = (int)(X.Kb[u] & 0xffffffff); }
                    } else if (lane == 0) {
                        unlink_row(X, cand, kk);
                        unlink_col(X, cand, kk);
                    }
                    __syncwarp();
                    leader_from_slot(X, ws, cand, L, Ld, freeTop, ovfFreeTop);
                }
            }
        }
        __syncwarp();
    }
    if (lane == 0) {
        I->n_ops = nop;
        I->n_members = nmem;
        if (err) I->status = err;
        else if (nmem != I->n_steps) I->status = RR_ERR_INTERNAL;
        else if (overflow) I->status = RR_ERR_CAPACITY;
    }
}

// ------------------------------------------------- small-grid simulation
//
// Alg. 4 for one small instance with the ready set in warp registers. At most
// SMALL_CAP moves may be ready at once: two per lane, slot j = 32 p + lane of
// plane p, kept sorted by move id, so that slot 0 holds the leader (the
// lowest unfinished id) and a ballot in slot order lists candidates in id
// order. Every segment is recomputed from the registers: the batch is the
// leader plus every ready move of its direction on its row (set A) or on its
// column (set B), whichever holds the lower id (the same rule as sim_body);
// the segment ends at the first leg end of a batch move or where the leader
// reaches a row (vertical moves) or column (horizontal ones) holding a ready
// move of its direction. Finishing moves release their successors (in-degrees
// in shared memory) and the ready set is re-sorted through shared memory.
// The move records are staged in shared memory first. An instance with more
// than SMALL_MAX_MOVES moves, or more than SMALL_CAP ready at once, is left to
// sim_body (status RR_SIM_RETRY: its wide pass redoes it from the start).
constexpr int SMALL_CAP = 64;
constexpr int SMALL_MAX_MOVES = 2048;
constexpr int SMALL_SBUF = 128;   // successor entries released per round

__host__ __device__ inline size_t small_smem_bytes()
{
    return 32ull * SMALL_MAX_MOVES + 4ull * SMALL_MAX_MOVES +      // records, in-degrees
           16ull * SMALL_CAP + 4ull * SMALL_CAP +                  // re-sort staging, sorted survivor ids
           4ull * (SMALL_CAP + 32) + 4ull * SMALL_SBUF + 4ull * (SMALL_CAP + 2);   // new ids, successors, batch
}

struct SmallSlot { int32_t id, key, rem, dst; };

__device__ __forceinline__ SmallSlot small_from_rec(int id, int4 r)
{
    const int sr = r.x & 0xffff, sc = r.x >> 16, dr = r.y & 0xffff, dc = r.y >> 16;
    const int d = dc != sc ? (dc > sc ? 3 : 2) : (dr > sr ? 1 : 0);
    return SmallSlot{id, key_of(sr, sc, d), dc != sc ? iabs(dc - sc) : iabs(dr - sr), dr};
}

// Returns with I->status unchanged (done), RR_SIM_RETRY (left to sim_body) or
// an error status. One warp; `sm` is this warp's shared memory.
__device__ inline void sim_small(rr_instance *I, JobWS &ws, char *sm)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    if (!live(I)) return;
    const int k = (int)I->n_moves;
    if (k == 0) { if (lane == 0) { I->n_ops = 0; I->n_members = 0; } return; }
    if (k > SMALL_MAX_MOVES) { if (lane == 0) I->status = RR_SIM_RETRY; return; }
    int4 *recs = (int4 *)sm;                                   // 2 per move: geometry, first successors
    int32_t *indeg = (int32_t *)(recs + 2 * SMALL_MAX_MOVES);
    SmallSlot *stage = (SmallSlot *)(indeg + SMALL_MAX_MOVES);
    int32_t *survIds = (int32_t *)(stage + SMALL_CAP);
    int32_t *newIds = survIds + SMALL_CAP;
    int32_t *sbuf = newIds + SMALL_CAP + 32;
    int32_t *bat = sbuf + SMALL_SBUF;
    for (int i = lane; i < 2 * k; i += 32) recs[i] = ws.rec[i];
    for (int i = lane; i < k; i += 32) indeg[i] = ws.indeg[i];
    __syncwarp();

    // the initially ready moves, sorted by id
    const int n0 = ws.ready0[k];
    if (n0 > SMALL_CAP) { if (lane == 0) I->status = RR_SIM_RETRY; return; }
    for (int i = lane; i < n0; i += 32) newIds[i] = ws.ready0[i];
    __syncwarp();
    SmallSlot S0{INTMAX, 0, 0, 0}, S1{INTMAX, 0, 0, 0};
    for (int i = lane; i < n0; i += 32) {
        const int id = newIds[i];
        int r = 0;
        for (int j = 0; j < n0; ++j) r += newIds[j] < id;
        stage[r] = small_from_rec(id, recs[2 * id]);
    }
    __syncwarp();
    if (lane < n0) S0 = stage[lane];
    if (32 + lane < n0) S1 = stage[32 + lane];
    __syncwarp();

    const int64_t cap_ops = I->cap_ops, cap_mem = I->cap_members;
    rr_op *ops = I->ops;
    int32_t *mem = I->members;
    int64_t nop = 0, nmem = 0;
    int overflow = 0, err = 0, done = 0;
    const int64_t guard_max = g_guard_cap > 0 ? g_guard_cap : I->n_steps + 2ll * k + 16;
    for (int64_t guard = 0;; ++guard) {
        if (guard >= guard_max) { err = RR_ERR_TIMEOUT; break; }
        const int Lid = __shfl_sync(FULL, S0.id, 0);
        if (Lid == INTMAX) break;
        const int Lkey = __shfl_sync(FULL, S0.key, 0);
        const int d = key_d(Lkey), lr = key_r(Lkey), lc = key_c(Lkey);
        const bool vert = d < 2;
        const int sgn = (d == 1 || d == 3) ? 1 : -1;
        // candidates: ready moves of direction d, the leader excluded
        const bool same0 = S0.id != INTMAX && key_d(S0.key) == d && lane != 0;
        const bool same1 = S1.id != INTMAX && key_d(S1.key) == d;
        const unsigned bR0 = __ballot_sync(FULL, same0 && key_r(S0.key) == lr);
        const unsigned bC0 = __ballot_sync(FULL, same0 && key_c(S0.key) == lc);
        const unsigned bR1 = __ballot_sync(FULL, same1 && key_r(S1.key) == lr);
        const unsigned bC1 = __ballot_sync(FULL, same1 && key_c(S1.key) == lc);
        unsigned m0 = 0u, m1 = 0u;
        if (bR0 | bC0) {
            const int f = __ffs(bR0 | bC0) - 1;
            const bool row = (bR0 >> f) & 1u;
            m0 = row ? bR0 : bC0;
            m1 = row ? bR1 : bC1;
        } else if (bR1 | bC1) {
            const int f = __ffs(bR1 | bC1) - 1;
            const bool row = (bR1 >> f) & 1u;
            m1 = row ? bR1 : bC1;
        }
        const bool in0 = lane == 0 || ((m0 >> lane) & 1u), in1 = (m1 >> lane) & 1u;
        const int ns = 1 + __popc(m0) + __popc(m1);
        // segment length: the first leg end in the batch, the nearest ready
        // move of direction d on a line ahead of the leader
        auto limit = [&](const SmallSlot &S, bool inB, bool same) {
            if (inB) return S.rem;
            if (same) {
                const int dist = (vert ? key_r(S.key) - lr : key_c(S.key) - lc) * sgn;
                if (dist > 0) return dist;
            }
            return INTMAX;
        };
        const int kseg = __reduce_min_sync(FULL, min(limit(S0, in0, same0), limit(S1, in1, same1)));
        if (kseg < 1 || kseg == INTMAX) { err = RR_ERR_INTERNAL; break; }
        // kseg identical batches: ids in rank order (leader first, then slot order)
        const int64_t addm = (int64_t)kseg * ns;
        if (!overflow && nop + kseg <= cap_ops && nmem + addm <= cap_mem) {
            for (int i = lane; i < kseg; i += 32) ops[nop + i] = rr_op{d, (int32_t)(nmem + (int64_t)i * ns), ns};
            // the batch's ids in rank order: the leader, then the members in
            // slot (id) order
            if (in0) bat[lane == 0 ? 0 : 1 + __popc(m0 & lt)] = S0.id;
            if (in1) bat[1 + __popc(m0) + __popc(m1 & lt)] = S1.id;
            __syncwarp();
            if (ns <= 32) {
                // lane r writes the r-th member of every batch of the segment
                const int v = lane < ns ? bat[lane] : 0;
                if (lane < ns)
                    for (int i = 0; i < kseg; ++i) mem[nmem + (int64_t)i * ns + lane] = v;
                __syncwarp();
            } else {
                int u = small_mod(lane, ns);
                const int step = small_mod(32, ns);
                for (int64_t i = lane; i < addm; i += 32) {
                    mem[nmem + i] = bat[u];
                    u += step;
                    if (u >= ns) u -= ns;
                }
                __syncwarp();
            }
        } else {
            overflow = 1;
        }
        nop += kseg;
        nmem += addm;
        // advance the batch; at a leg end a move turns toward its
        // destination row or finishes there
        bool fin0 = false, fin1 = false;
        auto advance = [&](SmallSlot &S, bool inB) {
            if (!inB) return false;
            int r = key_r(S.key), c = key_c(S.key), dd = key_d(S.key);
            if (dd == 0) r -= kseg; else if (dd == 1) r += kseg; else if (dd == 2) c -= kseg; else c += kseg;
            S.rem -= kseg;
            if (S.rem == 0) {
                if (r == S.dst) { S.key = key_of(r, c, dd); return true; }
                dd = S.dst > r ? 1 : 0;
                S.rem = iabs(S.dst - r);
            }
            S.key = key_of(r, c, dd);
            return false;
        };
        fin0 = advance(S0, in0);
        fin1 = advance(S1, in1);
        const unsigned f0 = __ballot_sync(FULL, fin0), f1 = __ballot_sync(FULL, fin1);
        if (!(f0 | f1)) continue;
        done += __popc(f0) + __popc(f1);
        // release the finished moves' successors, one finished move at a time
        // (lane e takes successor e); newly ready ids go to newIds
        int nn = 0;
        for (unsigned fm0 = f0, fm1 = f1; fm0 | fm1;) {
            int src, pl;
            if (fm0) { src = __ffs(fm0) - 1; fm0 &= fm0 - 1; pl = 0; }
            else { src = __ffs(fm1) - 1; fm1 &= fm1 - 1; pl = 1; }
            const int a0 = __shfl_sync(FULL, S0.id, src), a1 = __shfl_sync(FULL, S1.id, src);
            const int fid = pl ? a1 : a0;
            const int4 g = recs[2 * fid];
            const int32_t *s4 = (const int32_t *)&recs[2 * fid + 1];
            for (int e0 = 0; e0 < g.z; e0 += 32) {
                const int e = e0 + lane;
                int ready = -1;
                if (e < g.z) {
                    const int v = e < 4 ? s4[e] : ws.succ[g.w + e - 4];
                    const int sid = v & SUCC_ID;
                    if ((v & SUCC_SINGLE) || atomicSub(&indeg[sid], 1) == 1) ready = sid;
                }
                const unsigned bal = __ballot_sync(FULL, ready >= 0);
                if (ready >= 0 && nn + __popc(bal & lt) < 32) newIds[nn + __popc(bal & lt)] = ready;
                nn += __popc(bal);
            }
        }
        // the ready set again, sorted: survivors keep their order, newly ready
        // moves go between them by id
        const bool sv0 = S0.id != INTMAX && !fin0, sv1 = S1.id != INTMAX && !fin1;
        const unsigned b0v = __ballot_sync(FULL, sv0), b1v = __ballot_sync(FULL, sv1);
        const int nsv = __popc(b0v) + __popc(b1v);
        if (nn > 32 || nsv + nn > SMALL_CAP) { if (lane == 0) I->status = RR_SIM_RETRY; return; }
        __syncwarp();
        const int myNew = lane < nn ? newIds[lane] : INTMAX;
        int c0 = 0, c1 = 0, posNew = 0;
        for (int t = 0; t < nn; ++t) {
            const int id = __shfl_sync(FULL, myNew, t);
            const int below = __popc(__ballot_sync(FULL, sv0 && S0.id < id)) +
                              __popc(__ballot_sync(FULL, sv1 && S1.id < id)) +
                              __popc(__ballot_sync(FULL, myNew < id));
            if (lane == t) posNew = below;
            c0 += sv0 && id < S0.id;
            c1 += sv1 && id < S1.id;
        }
        if (sv0) stage[__popc(b0v & lt) + c0] = S0;
        if (sv1) stage[__popc(b0v) + __popc(b1v & lt) + c1] = S1;
        if (lane < nn) stage[posNew] = small_from_rec(myNew, recs[2 * myNew]);
        __syncwarp();
        const int T = nsv + nn;
        S0 = lane < T ? stage[lane] : SmallSlot{INTMAX, 0, 0, 0};
        S1 = 32 + lane < T ? stage[32 + lane] : SmallSlot{INTMAX, 0, 0, 0};
        __syncwarp();
    }
    if (lane == 0) {
        I->n_ops = nop;
        I->n_members = nmem;
        if (err) I->status = err;
        else if (done != k || nmem != I->n_steps) I->status = RR_ERR_INTERNAL;
        else if (overflow) I->status = RR_ERR_CAPACITY;
    }
}


} // namespace rrk
