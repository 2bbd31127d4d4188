// rr_batch.cu -- the batching routine (arXiv 2504.06182, Alg. 2 with the
// local constraint set of Sec. IV) on the GPU.
//
// Gamma (Sec. IV, "Input to the batching routine"): move b depends on every
// earlier move whose path shares a vertex with it. It is enough to keep, for
// every vertex, the immediately preceding path through it; a move is ready
// once all of those have finished. The kernels below build, per vertex, the
// list of paths through it in id order, and from it the de-duplicated
// successor lists and in-degrees.
//
// Alg. 2 itself runs as an event-driven simulation, one warp per instance.
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
#include "rr_internal.cuh"

namespace rrk {

__device__ __forceinline__ bool live(const rr_instance *I) { return I->status == RR_OK; }

// Chunked block-wide exclusive scan of v[0..len) in place; returns the total.
// Every thread of the block must call it.
__device__ long long block_exclusive_scan(int32_t *v, int len, long long *s_tmp /* >= 33 */)
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

// Position of vertex (r, c) along move p (row first, then column).
__device__ __forceinline__ int path_pos(const rr_move &p, int r, int c)
{
    const int hl = iabs(p.dst_col - p.src_col);
    if (r == p.src_row) {
        const int t = iabs(c - p.src_col);
        if (t <= hl && ((c - p.src_col) * (p.dst_col - p.src_col) >= 0)) return t;
    }
    return hl + iabs(r - p.src_row);
}

// ----------------------------------------------------------- set-up pass
// One block per instance: check the moves, count path vertices, allocate.
__global__ void k_bsetup(rr_instance *inst, JobWS *wsv, int count, Arena A)
{
    __shared__ long long s_tmp[34];
    __shared__ int s_bad;
    const int q = blockIdx.x;
    if (q >= count) return;
    rr_instance *I = &inst[q];
    if (!live(I)) return;
    JobWS &ws = wsv[q];
    const int m = I->m, n = I->n;
    const int64_t k = I->n_moves;
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
            ws.cellCnt = (int32_t *)arena_alloc(A, 4ull * (cells + 1), &ok);
            ws.cellCur = (int32_t *)arena_alloc(A, 4ull * cells, &ok);
            ws.cover = (int32_t *)arena_alloc(A, 4ull * (tp + 1), &ok);
            ws.nextAt = (int32_t *)arena_alloc(A, 4ull * (tp + 1), &ok);
            ws.succOff = (int32_t *)arena_alloc(A, 4ull * (k + 1), &ok);
            ws.indeg = (int32_t *)arena_alloc(A, 4ull * (k + 1), &ok);
            ws.rec = (int4 *)arena_alloc(A, 16ull * (k + 1), &ok);
            ws.succ4 = (int4 *)arena_alloc(A, 16ull * (k + 1), &ok);
            ws.ready0 = (int32_t *)arena_alloc(A, 4ull * (k + 1) + 16, &ok);
            ws.slotOvf = arena_alloc(A, 64ull * (k + 1), &ok);
            ws.succ = nullptr; ws.E = 0;
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
    const long long cells = (long long)m * n;
    for (long long v = threadIdx.x; v < cells; v += blockDim.x) { ws.cellCnt[v] = 0; ws.cellCur[v] = 0; }
    __syncthreads();
    const long long tot = block_exclusive_scan(ws.pairOff, (int)k, s_tmp);
    if (threadIdx.x == 0) ws.pairOff[k] = (int32_t)tot;
}

// Vertex counts per cell.
__global__ void k_bcount(rr_instance *inst, JobWS *wsv, int count)
{
    const int q = blockIdx.y;
    if (q >= count) return;
    const rr_instance *I = &inst[q];
    if (!live(I)) return;
    JobWS &ws = wsv[q];
    const int n = I->n;
    const int64_t k = I->n_moves;
    for (int64_t b = blockIdx.x * blockDim.x + threadIdx.x; b < k; b += (int64_t)gridDim.x * blockDim.x) {
        const rr_move p = I->moves[b];
        const int len = iabs(p.dst_col - p.src_col) + iabs(p.dst_row - p.src_row);
        for (int t = 0; t <= len; ++t) {
            int r, c; path_cell(p.src_row, p.src_col, p.dst_row, p.dst_col, t, &r, &c);
            atomicAdd(&ws.cellCnt[(size_t)r * n + c], 1);
        }
    }
}

__global__ void k_bscan_cells(rr_instance *inst, JobWS *wsv, int count)
{
    __shared__ long long s_tmp[34];
    const int q = blockIdx.x;
    if (q >= count) return;
    rr_instance *I = &inst[q];
    if (!live(I)) return;
    JobWS &ws = wsv[q];
    const int cells = I->m * I->n;
    const long long tot = block_exclusive_scan(ws.cellCnt, cells, s_tmp);
    if (threadIdx.x == 0) {
        ws.cellCnt[cells] = (int32_t)tot;
        if (tot != ws.P) I->status = RR_ERR_INTERNAL;
    }
}

__global__ void k_bfill(rr_instance *inst, JobWS *wsv, int count)
{
    const int q = blockIdx.y;
    if (q >= count) return;
    const rr_instance *I = &inst[q];
    if (!live(I)) return;
    JobWS &ws = wsv[q];
    const int n = I->n;
    const int64_t k = I->n_moves;
    for (int64_t b = blockIdx.x * blockDim.x + threadIdx.x; b < k; b += (int64_t)gridDim.x * blockDim.x) {
        const rr_move p = I->moves[b];
        const int len = iabs(p.dst_col - p.src_col) + iabs(p.dst_row - p.src_row);
        for (int t = 0; t <= len; ++t) {
            int r, c; path_cell(p.src_row, p.src_col, p.dst_row, p.dst_col, t, &r, &c);
            const size_t v = (size_t)r * n + c;
            ws.cover[ws.cellCnt[v] + atomicAdd(&ws.cellCur[v], 1)] = (int32_t)b;
        }
    }
}

// Per cell: order its paths by id, then record for each path the next path
// through this cell (or -1) at the path's own vertex index.
__global__ void k_bsort(rr_instance *inst, JobWS *wsv, int count)
{
    const int q = blockIdx.y;
    if (q >= count) return;
    const rr_instance *I = &inst[q];
    if (!live(I)) return;
    JobWS &ws = wsv[q];
    const int n = I->n;
    const long long cells = (long long)I->m * n;
    for (long long v = blockIdx.x * blockDim.x + threadIdx.x; v < cells; v += (long long)gridDim.x * blockDim.x) {
        const int lo = ws.cellCnt[v], hi = ws.cellCnt[v + 1];
        if (hi == lo) continue;
        int32_t *L = ws.cover + lo;
        for (int i = 1; i < hi - lo; ++i) {
            const int32_t x = L[i];
            int j = i - 1;
            while (j >= 0 && L[j] > x) { L[j + 1] = L[j]; --j; }
            L[j + 1] = x;
        }
        const int r = (int)(v / n), c = (int)(v % n);
        for (int i = 0; i < hi - lo; ++i) {
            const int32_t a = L[i];
            const rr_move p = I->moves[a];
            ws.nextAt[ws.pairOff[a] + path_pos(p, r, c)] = (i + 1 < hi - lo) ? L[i + 1] : -1;
        }
    }
}

// Distinct successors of one path, in first-occurrence order.
template <class Emit>
__device__ int distinct_succ(const int32_t *seq, int len, Emit emit)
{
    int cnt = 0;
    int32_t buf[16];
    int32_t last = -1;
    for (int t = 0; t < len; ++t) {
        const int32_t v = seq[t];
        if (v < 0 || v == last) continue;
        last = v;
        bool seen = false;
        const int lim = cnt < 16 ? cnt : 16;
        for (int u = 0; u < lim; ++u) if (buf[u] == v) { seen = true; break; }
        if (!seen && cnt >= 16)
            for (int u = 0; u < t; ++u) if (seq[u] == v) { seen = true; break; }
        if (seen) continue;
        if (cnt < 16) buf[cnt] = v;
        emit(cnt, v);
        ++cnt;
    }
    return cnt;
}

__global__ void k_bsucc_count(rr_instance *inst, JobWS *wsv, int count)
{
    const int q = blockIdx.y;
    if (q >= count) return;
    const rr_instance *I = &inst[q];
    if (!live(I)) return;
    JobWS &ws = wsv[q];
    const int64_t k = I->n_moves;
    for (int64_t b = blockIdx.x * blockDim.x + threadIdx.x; b < k; b += (int64_t)gridDim.x * blockDim.x) {
        const int lo = ws.pairOff[b], hi = ws.pairOff[b + 1];
        ws.succOff[b] = distinct_succ(ws.nextAt + lo, hi - lo, [](int, int32_t) {});
    }
}

__global__ void k_bsucc_scan(rr_instance *inst, JobWS *wsv, int count, Arena A)
{
    __shared__ long long s_tmp[34];
    const int q = blockIdx.x;
    if (q >= count) return;
    rr_instance *I = &inst[q];
    if (!live(I)) return;
    JobWS &ws = wsv[q];
    const int k = (int)I->n_moves;
    const long long E = block_exclusive_scan(ws.succOff, k, s_tmp);
    if (threadIdx.x == 0) {
        ws.succOff[k] = (int32_t)E;
        ws.E = E;
        bool ok = true;
        ws.succ = (int32_t *)arena_alloc(A, 4ull * (E + 1), &ok);
        if (!ok) I->status = RR_ERR_WORKSPACE;
    }
}

__global__ void k_bsucc_fill(rr_instance *inst, JobWS *wsv, int count)
{
    const int q = blockIdx.y;
    if (q >= count) return;
    const rr_instance *I = &inst[q];
    if (!live(I)) return;
    JobWS &ws = wsv[q];
    const int64_t k = I->n_moves;
    for (int64_t b = blockIdx.x * blockDim.x + threadIdx.x; b < k; b += (int64_t)gridDim.x * blockDim.x) {
        const int lo = ws.pairOff[b], hi = ws.pairOff[b + 1];
        int32_t *out = ws.succ + ws.succOff[b];
        int32_t *indeg = ws.indeg;
        distinct_succ(ws.nextAt + lo, hi - lo, [&](int u, int32_t s) { out[u] = s; atomicAdd(&indeg[s], 1); });
    }
}

// Per-move records for the simulation: packed geometry, successor count and
// the first four successors (flagged when the successor has no other
// predecessor); later successors are flagged in place. Moves without
// predecessors are listed as initially ready.
__global__ void k_brec(rr_instance *inst, JobWS *wsv, int count)
{
    const int q = blockIdx.y;
    if (q >= count) return;
    const rr_instance *I = &inst[q];
    if (!live(I)) return;
    JobWS &ws = wsv[q];
    const int64_t k = I->n_moves;
    for (int64_t b = blockIdx.x * blockDim.x + threadIdx.x; b < k; b += (int64_t)gridDim.x * blockDim.x) {
        const rr_move p = I->moves[b];
        const int lo = ws.succOff[b], hi = ws.succOff[b + 1];
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
        ws.rec[b] = r;
        ws.succ4[b] = make_int4(v[0], v[1], v[2], v[3]);
        if (ws.indeg[b] == 0) ws.ready0[atomicAdd(&ws.ready0[k], 1)] = (int32_t)b;
    }
}

// ---------------------------------------------------------- simulation
//
// The ready moves live in a slot table (structure of arrays). Slots below
// the shared-memory capacity are in shared memory, the rest in a global
// overflow area with the same layout. Per-(direction, row) and
// per-(direction, column) counters of ready moves (the leader included) tell
// in O(1) whether the leader's row and column hold other moves of its
// direction; if not, the leader moves alone until the next pickup, found in
// bitmaps of non-empty rows (vertical directions) and columns (horizontal
// ones). Otherwise one warp-wide pass over the slot table collects both
// candidate lines (ballot compaction), their smallest ids, their shortest
// remaining straight legs and the nearest waiting move the leader's line
// will reach.

constexpr int MAPN = 1024;      // id -> slot cache for finding the next leader
constexpr int SBUF = 512;       // successor entries released per round
constexpr int KEY_LIVE = 1 << 22;
constexpr int INTMAX = 0x7fffffff;

struct SlotSoA {
    int32_t *key;     // row | col << 10 | dir << 20 | KEY_LIVE; 0 when free
    int32_t *id;      // move id, INT_MAX when free
    int32_t *g0, *g1; // src_row | src_col << 16, dst_row | dst_col << 16
    int32_t *t;       // elementary steps done
    int32_t *legEnd;  // t at the end of the current straight leg
    int32_t *nsucc, *ovf;
    int4 *s4;         // first four successors
};

struct Sim {
    SlotSoA sm, gm;
    int C, m, n, Wm, Wn;
    int32_t *freeStk;
    int32_t *map;
    int32_t *rowCnt, *colCnt;   // [4][m], [4][n]
    uint32_t *rowBits, *colBits;  // [2][Wm] for directions 0, 1; [2][Wn] for 2, 3
    long long *MkA, *MkB;       // candidate lines: id << 32 | slot
    int32_t *M;                 // member slots of the current batch, sorted by id
    int32_t *sbuf;
};

#define SLOTF(X, f, i) (*((i) < (X).C ? &(X).sm.f[(i)] : &(X).gm.f[(i) - (X).C]))

__device__ __forceinline__ int key_of(int r, int c, int d) { return r | (c << 10) | (d << 20) | KEY_LIVE; }

// Position, direction and remaining straight leg after t steps of a move.
__device__ __forceinline__ void move_pos(int g0, int g1, int t, int *r, int *c, int *d, int *rem, int *len)
{
    const int sr = g0 & 0xffff, sc = g0 >> 16, dr = g1 & 0xffff, dc = g1 >> 16;
    const int hl = iabs(dc - sc);
    *len = hl + iabs(dr - sr);
    if (t < hl) { *d = dc > sc ? 3 : 2; *r = sr; *c = sc + (dc > sc ? t : -t); *rem = hl - t; }
    else { const int v = t - hl; *d = dr > sr ? 1 : 0; *r = sr + (dr > sr ? v : -v); *c = dc; *rem = *len - t; }
}

__device__ __forceinline__ int warp_min(int v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v = min(v, __shfl_xor_sync(FULL, v, o));
    return v;
}

// Add delta (+1 or -1) to the line counters of a live key and keep the
// pickup bitmaps equal to "counter > 0". Within one warp step all updates
// must have the same sign.
__device__ __forceinline__ void cnt_add(const Sim &X, int key, int delta)
{
    const int r = key & 1023, c = (key >> 10) & 1023, d = (key >> 20) & 3;
    const int o1 = atomicAdd(&X.rowCnt[d * X.m + r], delta);
    const int o2 = atomicAdd(&X.colCnt[d * X.n + c], delta);
    if (d < 2) {
        if (delta > 0 && o1 == 0) atomicOr(&X.rowBits[d * X.Wm + (r >> 5)], 1u << (r & 31));
        if (delta < 0 && o1 == 1) atomicAnd(&X.rowBits[d * X.Wm + (r >> 5)], ~(1u << (r & 31)));
    } else {
        if (delta > 0 && o2 == 0) atomicOr(&X.colBits[(d - 2) * X.Wn + (c >> 5)], 1u << (c & 31));
        if (delta < 0 && o2 == 1) atomicAnd(&X.colBits[(d - 2) * X.Wn + (c >> 5)], ~(1u << (c & 31)));
    }
}

// First i in 1..maxq with bit (pos + i*delta) set, or 0.
__device__ int bit_scan(const uint32_t *b, int limit, int pos, int delta, int maxq)
{
    for (int i = 1; i <= maxq; ++i) {
        const int x = pos + i * delta;
        if (x < 0 || x >= limit) return 0;
        const uint32_t w = b[x >> 5];
        if (w == 0u) { i = delta > 0 ? ((x | 31) - pos) : (pos - (x & ~31)); continue; }
        if ((w >> (x & 31)) & 1u) return i;
    }
    return 0;
}

// Lowest move id held in slots [0, hi) and its slot (warp-cooperative).
__device__ int lowest_slot(const Sim &X, int hi)
{
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
__device__ void warp_sort64(long long *a, int n)
{
    const int lane = threadIdx.x & 31;
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
__device__ __forceinline__ int alloc_slot(const Sim &X, int rank, int cnt, int &freeTop, int &ovfUsed, int &hi,
                                          int kmax, int *err)
{
    int si = -1;
    const int fromStack = min(cnt, freeTop);
    if (rank < fromStack) si = X.freeStk[freeTop - 1 - rank];
    else if (rank < cnt) si = X.C + ovfUsed + (rank - fromStack);
    freeTop -= fromStack;
    ovfUsed += cnt - fromStack;
    if (ovfUsed > kmax) *err = RR_ERR_INTERNAL;
    int top = si + 1;
#pragma unroll
    for (int o = 16; o; o >>= 1) top = max(top, __shfl_xor_sync(FULL, top, o));
    hi = max(hi, top);
    return si;
}

__device__ __forceinline__ void fill_slot(const Sim &X, int si, int id, int4 r, int4 s4)
{
    int rr, cc, d, rem, len;
    move_pos(r.x, r.y, 0, &rr, &cc, &d, &rem, &len);
    const int key = key_of(rr, cc, d);
    SLOTF(X, key, si) = key;
    SLOTF(X, id, si) = id;
    SLOTF(X, g0, si) = r.x;
    SLOTF(X, g1, si) = r.y;
    SLOTF(X, t, si) = 0;
    SLOTF(X, legEnd, si) = rem;
    SLOTF(X, nsucc, si) = r.z;
    SLOTF(X, ovf, si) = r.w;
    SLOTF(X, s4, si) = s4;
    X.map[id & (MAPN - 1)] = si;
    cnt_add(X, key, +1);
}

__global__ void k_sim(rr_instance *inst, JobWS *wsv, int count, int slotCap, int lineCap)
{
    extern __shared__ int4 smem_i4[];
    const int q = blockIdx.x;
    if (q >= count) return;
    rr_instance *I = &inst[q];
    if (!live(I)) return;
    JobWS &ws = wsv[q];
    const int k = (int)I->n_moves;
    const int m = I->m, n = I->n;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    if (k == 0) { if (lane == 0) { I->n_ops = 0; I->n_members = 0; } return; }

    // shared-memory layout (mirrored by the launcher's size computation)
    Sim X;
    X.C = slotCap; X.m = m; X.n = n; X.Wm = (m + 31) >> 5; X.Wn = (n + 31) >> 5;
    const int lbuf = 2 * (lineCap + 2);
    X.sm.s4 = smem_i4;
    X.MkA = (long long *)(X.sm.s4 + slotCap);
    X.MkB = X.MkA + lbuf;
    int32_t *p32 = (int32_t *)(X.MkB + lbuf);
    X.sm.key = p32; p32 += slotCap;
    X.sm.id = p32; p32 += slotCap;
    X.sm.g0 = p32; p32 += slotCap;
    X.sm.g1 = p32; p32 += slotCap;
    X.sm.t = p32; p32 += slotCap;
    X.sm.legEnd = p32; p32 += slotCap;
    X.sm.nsucc = p32; p32 += slotCap;
    X.sm.ovf = p32; p32 += slotCap;
    X.freeStk = p32; p32 += slotCap;
    X.map = p32; p32 += MAPN;
    X.M = p32; p32 += lineCap + 2;
    X.sbuf = p32; p32 += SBUF;
    X.rowCnt = p32; p32 += 4 * lineCap;
    X.colCnt = p32; p32 += 4 * lineCap;
    X.rowBits = (uint32_t *)p32; p32 += 2 * ((lineCap + 31) >> 5);
    X.colBits = (uint32_t *)p32;
    {   // overflow slots (global), same structure
        char *g = (char *)ws.slotOvf;
        const size_t K1 = (size_t)k + 1;
        X.gm.s4 = (int4 *)g;               g += 16 * K1;
        X.gm.key = (int32_t *)g;           g += 4 * K1;
        X.gm.id = (int32_t *)g;            g += 4 * K1;
        X.gm.g0 = (int32_t *)g;            g += 4 * K1;
        X.gm.g1 = (int32_t *)g;            g += 4 * K1;
        X.gm.t = (int32_t *)g;             g += 4 * K1;
        X.gm.legEnd = (int32_t *)g;        g += 4 * K1;
        X.gm.nsucc = (int32_t *)g;         g += 4 * K1;
        X.gm.ovf = (int32_t *)g;
    }
    for (int i = lane; i < slotCap; i += 32) { X.sm.key[i] = 0; X.sm.id[i] = INTMAX; X.freeStk[i] = slotCap - 1 - i; }
    for (int i = lane; i < MAPN; i += 32) X.map[i] = -1;
    for (int i = lane; i < 4 * m; i += 32) X.rowCnt[i] = 0;
    for (int i = lane; i < 4 * n; i += 32) X.colCnt[i] = 0;
    for (int i = lane; i < 2 * X.Wm; i += 32) X.rowBits[i] = 0u;
    for (int i = lane; i < 2 * X.Wn; i += 32) X.colBits[i] = 0u;
    int freeTop = slotCap, ovfUsed = 0, hi = 0, err = 0;
    __syncwarp();

    // moves without predecessors
    const int32_t *ready0 = ws.ready0;
    const int nready0 = ready0[k];
    for (int base = 0; base < nready0; base += 32) {
        const int cnt = min(32, nready0 - base);
        int id = -1;
        int4 r = make_int4(0, 0, 0, 0), s4 = r;
        if (lane < cnt) { id = ready0[base + lane]; r = ws.rec[id]; s4 = ws.succ4[id]; }
        const int si = alloc_slot(X, lane, cnt, freeTop, ovfUsed, hi, k, &err);
        if (lane < cnt) fill_slot(X, si, id, r, s4);
        __syncwarp();
    }

    const int64_t cap_ops = I->cap_ops, cap_mem = I->cap_members;
    rr_op *ops = I->ops;
    int32_t *mem = I->members;
    int64_t nop = 0, nmem = 0;
    int overflow = 0;
    int Ls = lowest_slot(X, hi);
    int L = Ls >= 0 ? SLOTF(X, id, Ls) : -1;
    if (L != 0) err = RR_ERR_INTERNAL;
    const int64_t guard_max = I->n_steps + 2ll * k + 16;
    int64_t guard = 0;

    while (!err && L < k) {
        if (++guard > guard_max) { err = RR_ERR_TIMEOUT; break; }
        int lr, lc, d, remL, lenL;
        move_pos(SLOTF(X, g0, Ls), SLOTF(X, g1, Ls), SLOTF(X, t, Ls), &lr, &lc, &d, &remL, &lenL);
        const int sgn = (d == 1 || d == 3) ? 1 : -1;
        const int othersA = X.rowCnt[d * m + lr] - 1, othersB = X.colCnt[d * n + lc] - 1;
        int kseg = remL, ns = 1;
        long long *Mk = X.MkA;
        if (othersA == 0 && othersB == 0) {
            // the leader alone until the next waiting move of its direction
            if (kseg > 1) {
                const int hit = d >= 2 ? bit_scan(X.colBits + (d - 2) * X.Wn, n, lc, sgn, kseg - 1)
                                       : bit_scan(X.rowBits + d * X.Wm, m, lr, sgn, kseg - 1);
                if (hit > 0) kseg = hit;
            }
        } else {
            int minA = INTMAX, minB = INTMAX, pickA = INTMAX, pickB = INTMAX, remA = INTMAX, remB = INTMAX;
            int cntA = 0, cntB = 0;
            auto visit = [&](int key, int id, int rem, int i) {
                const bool same = (key & KEY_LIVE) && ((key >> 20) & 3) == d && i != Ls;
                const int sr = key & 1023, sc = (key >> 10) & 1023;
                const bool inA = same && sr == lr, inB = same && sc == lc;
                if (inA) { minA = min(minA, id); remA = min(remA, rem); }
                if (inB) { minB = min(minB, id); remB = min(remB, rem); }
                const int dist = (d >= 2 ? sc - lc : sr - lr) * sgn;
                if (same && dist > 0) {
                    if (!inA) pickA = min(pickA, dist);
                    if (!inB) pickB = min(pickB, dist);
                }
                const unsigned bA = __ballot_sync(FULL, inA), bB = __ballot_sync(FULL, inB);
                const long long kv = ((long long)id << 32) | (unsigned)i;
                if (inA && cntA + __popc(bA & lt) < lbuf) X.MkA[cntA + __popc(bA & lt)] = kv;
                if (inB && cntB + __popc(bB & lt) < lbuf) X.MkB[cntB + __popc(bB & lt)] = kv;
                cntA += __popc(bA);
                cntB += __popc(bB);
            };
            const int hs = min(hi, X.C);
            int i0 = 0;
            for (; i0 + 128 <= hs; i0 += 128) {
                int kk[4], id[4], le[4], tt[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int i = i0 + 32 * u + lane;
                    kk[u] = X.sm.key[i]; id[u] = X.sm.id[i]; le[u] = X.sm.legEnd[i]; tt[u] = X.sm.t[i];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) visit(kk[u], id[u], le[u] - tt[u], i0 + 32 * u + lane);
            }
            for (; i0 < hi; i0 += 32) {
                const int i = i0 + lane;
                const bool ok = i < hi;
                const int key = ok ? SLOTF(X, key, i) : 0;
                const int id = ok ? SLOTF(X, id, i) : INTMAX;
                const int rem = ok ? SLOTF(X, legEnd, i) - SLOTF(X, t, i) : 0;
                visit(key, id, rem, i);
            }
            minA = warp_min(minA); minB = warp_min(minB);
            pickA = warp_min(pickA); pickB = warp_min(pickB);
            remA = warp_min(remA); remB = warp_min(remB);
            if (cntA > lineCap || cntB > lineCap) { err = RR_ERR_INTERNAL; break; }
            const bool useA = minA < minB;
            kseg = min(kseg, useA ? min(remA, pickA) : min(remB, pickB));
            Mk = useA ? X.MkA : X.MkB;
            const int cnt = useA ? cntA : cntB;
            __syncwarp();
            warp_sort64(Mk, cnt);
            for (int u = lane; u < cnt; u += 32) X.M[1 + u] = (int)(Mk[u] & 0xffffffff);
            ns = 1 + cnt;
        }
        if (lane == 0) X.M[0] = Ls;
        __syncwarp();
        if (kseg < 1) { err = RR_ERR_INTERNAL; break; }

        // kseg identical batches: the leader, then the line in ascending id
        const int64_t addm = (int64_t)kseg * ns;
        if (!overflow && nop + kseg <= cap_ops && nmem + addm <= cap_mem) {
            for (int i = lane; i < kseg; i += 32) ops[nop + i] = rr_op{d, (int32_t)(nmem + (int64_t)i * ns), ns};
            if (ns == 1) {
                for (int i = lane; i < kseg; i += 32) mem[nmem + i] = L;
            } else {
                int u = lane % ns;
                const int step = 32 % ns;
                for (int64_t i = lane; i < addm; i += 32) {
                    mem[nmem + i] = u == 0 ? L : (int)(Mk[u - 1] >> 32);
                    u += step;
                    if (u >= ns) u -= ns;
                }
            }
        } else {
            overflow = 1;
        }
        nop += kseg;
        nmem += addm;

        // advance every member; finished ones release their successors
        int leaderDone = 0;
        for (int u0 = 0; u0 < ns; u0 += 32) {
            const int u = u0 + lane;
            bool fin = false, act = u < ns;
            int si = -1, nsu = 0, newKey = 0, newLeg = 0, t = 0;
            if (act) {
                si = X.M[u];
                t = SLOTF(X, t, si) + kseg;
                int r_, c_, d_, rem, len;
                move_pos(SLOTF(X, g0, si), SLOTF(X, g1, si), t, &r_, &c_, &d_, &rem, &len);
                fin = t >= len;
                newKey = key_of(r_, c_, d_);
                newLeg = t + rem;
                cnt_add(X, SLOTF(X, key, si), -1);
            }
            __syncwarp();
            if (act) {
                SLOTF(X, t, si) = t;
                if (fin) nsu = SLOTF(X, nsucc, si);
                else { SLOTF(X, key, si) = newKey; SLOTF(X, legEnd, si) = newLeg; cnt_add(X, newKey, +1); }
            }
            if (u0 == 0 && __shfl_sync(FULL, (int)fin, 0)) leaderDone = 1;
            __syncwarp();
            // successor entries of the finished members, in rounds of SBUF
            const int off = warp_incl_scan(nsu) - nsu;
            const int total = __shfl_sync(FULL, off + nsu, 31);
            for (int base = 0; base < total; base += SBUF) {
                if (fin) {
                    const int4 s4 = SLOTF(X, s4, si);
                    const int ov = SLOTF(X, ovf, si);
                    for (int e = max(0, base - off); e < nsu && off + e < base + SBUF; ++e)
                        X.sbuf[off + e - base] = e == 0 ? s4.x : e == 1 ? s4.y : e == 2 ? s4.z : e == 3 ? s4.w
                                                                                              : ~(ov + e - 4);
                }
                __syncwarp();
                const int nb = min(SBUF, total - base);
                for (int b0 = 0; b0 < nb; b0 += 32) {
                    int ready = -1;
                    int4 r = make_int4(0, 0, 0, 0), s4 = r;
                    if (b0 + lane < nb) {
                        int32_t e = X.sbuf[b0 + lane];
                        if (e < 0) e = ws.succ[~e];
                        const int id = e & SUCC_ID;
                        r = ws.rec[id]; s4 = ws.succ4[id];     // fetched with the counter update
                        if ((e & SUCC_SINGLE) || atomicSub(&ws.indeg[id], 1) == 1) ready = id;
                    }
                    const unsigned bal = __ballot_sync(FULL, ready >= 0);
                    const int cnt = __popc(bal);
                    if (cnt) {
                        const int ns_ = alloc_slot(X, __popc(bal & lt), cnt, freeTop, ovfUsed, hi, k, &err);
                        if (ready >= 0) fill_slot(X, ns_, ready, r, s4);
                    }
                    __syncwarp();
                }
            }
            // free the finished members' slots (shared-memory ones are recycled)
            if (fin) {
                const int id = SLOTF(X, id, si);
                if (X.map[id & (MAPN - 1)] == si) X.map[id & (MAPN - 1)] = -1;
                SLOTF(X, key, si) = 0;
                SLOTF(X, id, si) = INTMAX;
            }
            const bool recyc = fin && si < X.C;
            const unsigned fb = __ballot_sync(FULL, recyc);
            if (recyc) X.freeStk[freeTop + __popc(fb & lt)] = si;
            freeTop += __popc(fb);
            __syncwarp();
        }
        if (leaderDone && !err) {
            // next leader: lowest id still held in a slot (usually L + 1)
            int cand = -1;
            const int nx = L + 1;
            if (nx < k) {
                const int si = X.map[nx & (MAPN - 1)];
                if (si >= 0 && SLOTF(X, id, si) == nx) cand = si;
            }
            if (cand < 0) cand = lowest_slot(X, hi);
            if (cand < 0) L = k;
            else { Ls = cand; L = SLOTF(X, id, Ls); }
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

} // namespace rrk
