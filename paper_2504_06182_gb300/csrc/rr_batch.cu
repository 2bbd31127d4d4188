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
            ws.pst = (int32_t *)arena_alloc(A, 4ull * PST_STRIDE * (k + 1) + 4ull * ((k + 32) / 32), &ok);
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
        int32_t *ps = ws.pst + PST_STRIDE * b;
        ps[0] = 0; ps[1] = -1; ps[2] = -1; ps[3] = -1; ps[4] = -1;
    }
    uint32_t *done = (uint32_t *)(ws.pst + PST_STRIDE * (k + 1));
    for (int64_t w = threadIdx.x; w < (k + 32) / 32; w += blockDim.x) done[w] = 0u;
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

// ---------------------------------------------------------- simulation

struct SimSmem {
    int32_t *rowHead;   // [4][m]
    int32_t *colHead;   // [4][n]
    uint32_t *rowBits;  // [2][Wm] dirs 0,1 : rows with a waiting move of that direction
    uint32_t *colBits;  // [2][Wn] dirs 2,3 : columns with a waiting move of that direction
    int32_t *S;         // batch members
    int m, n, Wm, Wn;
};

struct PathGeo {
    int sr, sc, dr, dc, len, hl;
};

__device__ __forceinline__ PathGeo load_geo(const rr_move *mv, int p)
{
    const rr_move x = mv[p];
    PathGeo g;
    g.sr = x.src_row; g.sc = x.src_col; g.dr = x.dst_row; g.dc = x.dst_col;
    g.hl = iabs(g.dc - g.sc);
    g.len = g.hl + iabs(g.dr - g.sr);
    return g;
}

__device__ __forceinline__ void geo_at(const PathGeo &g, int t, int *d, int *r, int *c, int *rem)
{
    if (t < g.hl) { *d = g.dc > g.sc ? 3 : 2; *r = g.sr; *c = g.sc + t * isgn(g.dc - g.sc); *rem = g.hl - t; }
    else { *d = g.dr > g.sr ? 1 : 0; *r = g.sr + (t - g.hl) * isgn(g.dr - g.sr); *c = g.dc; *rem = g.len - t; }
}

__device__ __forceinline__ void bit_set(uint32_t *b, int i) { b[i >> 5] |= 1u << (i & 31); }
__device__ __forceinline__ void bit_clr(uint32_t *b, int i) { b[i >> 5] &= ~(1u << (i & 31)); }

// Lists of waiting ready moves per (direction, row) and (direction, column).
__device__ void line_insert(SimSmem &S, int32_t *pst, int p, int d, int r, int c)
{
    int32_t *ps = pst + PST_STRIDE * p;
    int32_t *hr = &S.rowHead[d * S.m + r];
    ps[1] = -1; ps[2] = *hr;
    if (*hr >= 0) pst[PST_STRIDE * *hr + 1] = p;
    *hr = p;
    int32_t *hc = &S.colHead[d * S.n + c];
    ps[3] = -1; ps[4] = *hc;
    if (*hc >= 0) pst[PST_STRIDE * *hc + 3] = p;
    *hc = p;
    if (d < 2) bit_set(S.rowBits + d * S.Wm, r); else bit_set(S.colBits + (d - 2) * S.Wn, c);
}

__device__ void line_remove(SimSmem &S, int32_t *pst, int p, int d, int r, int c)
{
    int32_t *ps = pst + PST_STRIDE * p;
    const int rp = ps[1], rn = ps[2], cp = ps[3], cn = ps[4];
    if (rp >= 0) pst[PST_STRIDE * rp + 2] = rn; else S.rowHead[d * S.m + r] = rn;
    if (rn >= 0) pst[PST_STRIDE * rn + 1] = rp;
    if (cp >= 0) pst[PST_STRIDE * cp + 4] = cn; else S.colHead[d * S.n + c] = cn;
    if (cn >= 0) pst[PST_STRIDE * cn + 3] = cp;
    if (d < 2) { if (S.rowHead[d * S.m + r] < 0) bit_clr(S.rowBits + d * S.Wm, r); }
    else { if (S.colHead[d * S.n + c] < 0) bit_clr(S.colBits + (d - 2) * S.Wn, c); }
}

// First i in 1..maxq with bit (pos + i*delta) set, or 0.
__device__ int bit_scan(const uint32_t *b, int limit, int pos, int delta, int maxq)
{
    for (int i = 1; i <= maxq; ++i) {
        const int x = pos + i * delta;
        if (x < 0 || x >= limit) return 0;
        const uint32_t w = b[x >> 5];
        if (w == 0u) {
            // skip the rest of an empty word
            const int edge = delta > 0 ? ((x | 31) - pos) : (pos - (x & ~31));
            i = edge;
            continue;
        }
        if ((w >> (x & 31)) & 1u) return i;
    }
    return 0;
}

__global__ void k_sim(rr_instance *inst, JobWS *wsv, int count)
{
    extern __shared__ int32_t smem_i32[];
    const int q = blockIdx.x;
    if (q >= count) return;
    rr_instance *I = &inst[q];
    if (!live(I)) return;
    JobWS &ws = wsv[q];
    const int m = I->m, n = I->n;
    const int k = (int)I->n_moves;
    const int lane = threadIdx.x & 31;
    if (k == 0) { if (lane == 0) { I->n_ops = 0; I->n_members = 0; } return; }

    SimSmem S;
    S.m = m; S.n = n; S.Wm = (m + 31) >> 5; S.Wn = (n + 31) >> 5;
    S.rowHead = smem_i32;
    S.colHead = S.rowHead + 4 * m;
    S.rowBits = (uint32_t *)(S.colHead + 4 * n);
    S.colBits = S.rowBits + 2 * S.Wm;
    S.S = (int32_t *)(S.colBits + 2 * S.Wn);
    for (int i = lane; i < 4 * m; i += 32) S.rowHead[i] = -1;
    for (int i = lane; i < 4 * n; i += 32) S.colHead[i] = -1;
    for (int i = lane; i < 2 * S.Wm; i += 32) S.rowBits[i] = 0u;
    for (int i = lane; i < 2 * S.Wn; i += 32) S.colBits[i] = 0u;
    __syncwarp();

    int32_t *pst = ws.pst;
    uint32_t *done = (uint32_t *)(ws.pst + PST_STRIDE * (k + 1));
    const rr_move *mv = I->moves;
    const int32_t *indeg0 = ws.indeg;
    // initially ready moves (in-degree 0), inserted by lane 0 in id order
    for (int base = 0; base < k; base += 32) {
        const int b = base + lane;
        const unsigned bal = __ballot_sync(FULL, b < k && indeg0[b] == 0);
        if (lane == 0) {
            unsigned x = bal;
            while (x) {
                const int p = base + __ffs(x) - 1;
                x &= x - 1;
                const PathGeo g = load_geo(mv, p);
                int d, r, c, rem; geo_at(g, 0, &d, &r, &c, &rem);
                line_insert(S, pst, p, d, r, c);
            }
        }
        __syncwarp();
    }

    const int64_t cap_ops = I->cap_ops, cap_mem = I->cap_members;
    rr_op *ops = I->ops;
    int32_t *mem = I->members;
    int64_t nop = 0, nmem = 0;
    int overflow = 0, err = 0;

    // leader state (kept uniform across the warp via lane-0 broadcasts)
    int L = 0;
    PathGeo Lg = load_geo(mv, 0);
    int Lt = 0;
    if (lane == 0) {
        if (indeg0[0] != 0) err = RR_ERR_INTERNAL;
        int d, r, c, rem; geo_at(Lg, 0, &d, &r, &c, &rem);
        line_remove(S, pst, 0, d, r, c);
    }
    err = __shfl_sync(FULL, err, 0);
    const int64_t guard_max = I->n_steps + (int64_t)k + 16;
    int64_t guard = 0;

    while (!err && L < k) {
        if (++guard > guard_max) { err = RR_ERR_TIMEOUT; break; }
        int ns = 0, d = 0, kseg = 0;
        if (lane == 0) {
            int r, c, remL; geo_at(Lg, Lt, &d, &r, &c, &remL);
            // candidates on the leader's row (A) and column (B)
            // a line holds at most one token per trap: walks longer than that
            // mean a corrupted list and end the simulation with an error
            const int lineCap = max(m, n);
            int minA = 0x7fffffff, minB = 0x7fffffff, walk = 0;
            for (int p = S.rowHead[d * m + r]; p >= 0 && walk <= lineCap; p = pst[PST_STRIDE * p + 2], ++walk)
                minA = min(minA, p);
            for (int p = S.colHead[d * n + c]; p >= 0 && walk <= 2 * lineCap; p = pst[PST_STRIDE * p + 4], ++walk)
                minB = min(minB, p);
            if (walk > 2 * lineCap) err = RR_ERR_INTERNAL;
            S.S[0] = L; ns = 1;
            kseg = remL;
            if (!err && (minA != 0x7fffffff || minB != 0x7fffffff)) {
                const bool useA = minA < minB;
                for (int p = useA ? S.rowHead[d * m + r] : S.colHead[d * n + c]; p >= 0 && ns <= lineCap;
                     p = pst[PST_STRIDE * p + (useA ? 2 : 4)])
                    S.S[ns++] = p;
                for (int u = 1; u < ns; ++u) {
                    const int p = S.S[u];
                    const PathGeo g = load_geo(mv, p);
                    int dd, rr, cc, rem; geo_at(g, pst[PST_STRIDE * p], &dd, &rr, &cc, &rem);
                    kseg = min(kseg, rem);
                }
                for (int u = 1; u < ns; ++u) {
                    const int p = S.S[u];
                    const PathGeo g = load_geo(mv, p);
                    int dd, rr, cc, rem; geo_at(g, pst[PST_STRIDE * p], &dd, &rr, &cc, &rem);
                    line_remove(S, pst, p, dd, rr, cc);
                }
                // members in ascending id (insertion sort; batches are short)
                for (int u = 2; u < ns; ++u) {
                    const int x = S.S[u];
                    int v = u - 1;
                    while (v >= 1 && S.S[v] > x) { S.S[v + 1] = S.S[v]; --v; }
                    S.S[v + 1] = x;
                }
            }
            // a waiting move of direction d that the leader's line reaches
            if (kseg > 1) {
                int hit;
                if (d >= 2) hit = bit_scan(S.colBits + (d - 2) * S.Wn, n, c, d == 3 ? 1 : -1, kseg - 1);
                else hit = bit_scan(S.rowBits + d * S.Wm, m, r, d == 1 ? 1 : -1, kseg - 1);
                if (hit > 0) kseg = hit;
            }
        }
        ns = __shfl_sync(FULL, ns, 0);
        d = __shfl_sync(FULL, d, 0);
        kseg = __shfl_sync(FULL, kseg, 0);
        err = __shfl_sync(FULL, err, 0);
        __syncwarp();
        if (err) break;
        if (kseg < 1) { err = RR_ERR_INTERNAL; break; }
        // write kseg identical batches
        const int64_t addm = (int64_t)kseg * ns;
        if (!overflow && nop + kseg <= cap_ops && nmem + addm <= cap_mem) {
            for (int i = lane; i < kseg; i += 32) ops[nop + i] = rr_op{d, (int32_t)(nmem + (int64_t)i * ns), ns};
            if (ns == 1) {
                for (int i = lane; i < kseg; i += 32) mem[nmem + i] = L;
            } else {
                for (int64_t i = lane; i < addm; i += 32) mem[nmem + i] = S.S[i % ns];
            }
        } else {
            overflow = 1;
        }
        nop += kseg;
        nmem += addm;
        __syncwarp();
        // advance members, retire finished moves, reinsert the others
        int newL = L;
        if (lane == 0) {
            for (int u = 1; u < ns; ++u) {
                const int p = S.S[u];
                const PathGeo g = load_geo(mv, p);
                const int t = pst[PST_STRIDE * p] + kseg;
                pst[PST_STRIDE * p] = t;
                if (t >= g.len) {
                    done[p >> 5] |= 1u << (p & 31);
                    for (int e = ws.succOff[p]; e < ws.succOff[p + 1]; ++e) {
                        const int s = ws.succ[e];
                        if (atomicSub(&ws.indeg[s], 1) == 1) {
                            const PathGeo gs = load_geo(mv, s);
                            int dd, rr, cc, rem; geo_at(gs, pst[PST_STRIDE * s], &dd, &rr, &cc, &rem);
                            line_insert(S, pst, s, dd, rr, cc);
                        }
                    }
                } else {
                    int dd, rr, cc, rem; geo_at(g, t, &dd, &rr, &cc, &rem);
                    line_insert(S, pst, p, dd, rr, cc);
                }
            }
            Lt += kseg;
            if (Lt >= Lg.len) {
                pst[PST_STRIDE * L] = Lt;
                done[L >> 5] |= 1u << (L & 31);
                for (int e = ws.succOff[L]; e < ws.succOff[L + 1]; ++e) {
                    const int s = ws.succ[e];
                    if (atomicSub(&ws.indeg[s], 1) == 1) {
                        const PathGeo gs = load_geo(mv, s);
                        int dd, rr, cc, rem; geo_at(gs, pst[PST_STRIDE * s], &dd, &rr, &cc, &rem);
                        line_insert(S, pst, s, dd, rr, cc);
                    }
                }
                // next leader: lowest id not yet finished
                int nl = L + 1;
                while (nl < k) {
                    const uint32_t w = ~done[nl >> 5] & (0xffffffffu << (nl & 31));
                    if (w) { nl = (nl & ~31) + __ffs(w) - 1; break; }
                    nl = (nl & ~31) + 32;
                }
                newL = nl < k ? nl : k;
                if (newL < k) {
                    if (ws.indeg[newL] != 0) err = RR_ERR_INTERNAL;
                    Lg = load_geo(mv, newL);
                    Lt = pst[PST_STRIDE * newL];
                    int dd, rr, cc, rem; geo_at(Lg, Lt, &dd, &rr, &cc, &rem);
                    line_remove(S, pst, newL, dd, rr, cc);
                }
            }
        }
        __syncwarp();
        newL = __shfl_sync(FULL, newL, 0);
        err = __shfl_sync(FULL, err, 0);
        if (newL != L) {
            L = newL;
            if (L < k) {
                Lg.sr = __shfl_sync(FULL, Lg.sr, 0); Lg.sc = __shfl_sync(FULL, Lg.sc, 0);
                Lg.dr = __shfl_sync(FULL, Lg.dr, 0); Lg.dc = __shfl_sync(FULL, Lg.dc, 0);
                Lg.len = __shfl_sync(FULL, Lg.len, 0); Lg.hl = __shfl_sync(FULL, Lg.hl, 0);
            }
        }
        Lt = __shfl_sync(FULL, Lt, 0);
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
