// rr_bird.cu -- planning kernel of the bird algorithm (arXiv 2504.06182,
// Alg. 2, Sec. III.E).
//
// The column phase is red-rec's (k_colstats and k_emit_cols: every column of
// non-negative surplus solved by the exact 1D algorithm, columns outside the
// target columns pushed into their reservoir rows). What remains is
// sequential by definition: the unsolved columns are filled one after the
// other, left to right, each from every token of the grid at once, and each
// fill changes the tokens the next one sees. One block per grid runs that
// loop with the grid's reservoir rows resident in shared memory.
//
// The generalised 1D instance of receiver column j (Sec. III.E): an atom in a
// reservoir row v of a column at distance d sits on vertex v - d of column j
// above the band and on v + d below it, so that its Manhattan distance to any
// band trap of j is its distance along j. Tokens on one diagonal share a
// vertex. The vertices nearest the band are visited outward, layer by layer
// (layer k = vertex r0 - 1 - k above, r1 + k below; inside a layer the nearer
// column first, left before right): the first tokens met are the nearest,
// which is the order in which the optimal window takes them. The window
// itself is red-rec's split: a tokens from above, all band atoms of j, the
// rest from below, a of least total distance (largest a on ties), found by
// the discrete derivative of the convex cost.
#include "rr_internal.cuh"

namespace rrk {

// Token of a walk list: row in the upper 16 bits, column in the lower.
__device__ __forceinline__ int tok_row(int v) { return v >> 16; }
__device__ __forceinline__ int tok_col(int v) { return v & 0xffff; }

__device__ __forceinline__ int isqrt_floor(int g)
{
    int k = (int)sqrtf((float)g);
    while (k * k > g) --k;
    while ((k + 1) * (k + 1) <= g) ++k;
    return k;
}

// Collects, nearest first, up to `need` tokens of receiver j on one side of
// the band (one warp). Cell g of the walk is layer k = floor(sqrt(g)), index
// i = g - k*k in it: i = 0 is column j itself, i = 2d-1 column j-d, i = 2d
// column j+d, on row r0-1-k+d above the band or r1+k-d below it.
__device__ int bird_walk(const uint32_t *bits, int W, int m, int n, int r0, int r1, int j, bool top, int need,
                         int32_t *list)
{
    const int lane = threadIdx.x & 31;
    if (top ? r0 == 0 : r1 == m) return 0;
    const int dmax = max(j, n - 1 - j);
    const int kmax = top ? r0 - 1 + dmax : m - 1 - r1 + dmax;   // no cell beyond this layer
    int got = 0;
    for (int base = 0; got < need && isqrt_floor(base) <= kmax; base += 32) {
        const int g = base + lane;
        const int k = isqrt_floor(g);
        const int i = g - k * k;
        const int d = (i + 1) >> 1;
        const int col = d == 0 ? j : ((i & 1) ? j - d : j + d);
        const int row = top ? r0 - 1 - k + d : r1 + k - d;
        bool occ = false;
        if (k <= kmax && col >= 0 && col < n && row >= 0 && row < m)
            occ = (bits[(size_t)col * W + (row >> 5)] >> (row & 31)) & 1u;
        const unsigned bal = __ballot_sync(FULL, occ);
        const int rank = got + __popc(bal & ((1u << lane) - 1u));
        if (occ && rank < need) list[rank] = (row << 16) | col;
        got = min(need, got + __popc(bal));
    }
    return got;
}

__global__ void __launch_bounds__(64) k_bird(rr_instance *inst, JobWS *wsv, int count, int max_side)
{
    extern __shared__ uint32_t birdsm[];
    __shared__ int s_nt, s_nb, s_a, s_base, s_bad;
    const int q = blockIdx.x;
    if (q >= count) return;
    rr_instance *I = &inst[q];
    if (!live(I)) return;
    JobWS &ws = wsv[q];
    const int m = I->m, n = I->n, W = (m + 31) >> 5;
    const int r0 = I->rect.r0, r1 = I->rect.r1, c0 = I->rect.c0, c1 = I->rect.c1, h = r1 - r0;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    uint32_t *bits = birdsm;                                               // n * W words
    int32_t *topTok = (int32_t *)(birdsm + (size_t)max_side * ((max_side + 31) >> 5));
    int32_t *botTok = topTok + max_side;

    // Feasibility (total surplus, Sec. III.C) and the offsets of the column
    // units, in column order.
    if (wid == 0) {
        int tot = 0, carry = 0;
        for (int base = 0; base < n; base += 32) {
            const int c = base + lane;
            int v = 0;
            if (c < n) { v = ws.col[c].nmoves; tot += ws.col[c].sigma; }
            const int incl = warp_incl_scan(v);
            if (c < n) ws.unitOff[c] = carry + incl - v;
            carry += __shfl_sync(FULL, incl, 31);
        }
        tot = warp_sum(tot);
        if (lane == 0) {
            ws.unitOff[n] = carry;
            s_base = carry;
            s_bad = tot < 0;
        }
    }
    // Reservoir rows after the column phase: solved target columns keep the
    // atoms outside their window, outer columns with enough atoms fill every
    // reservoir trap, the others are untouched. Band rows are never read.
    for (int idx = tid; idx < n * W; idx += blockDim.x) {
        const int c = idx / W, w = idx - c * W;
        const ColInfo ci = ws.col[c];
        const uint32_t res = row_mask(w, 0, r0) | row_mask(w, r1, m);
        uint32_t x = ws.colbits[idx];
        if (ci.kind == KIND_OUTER_FULL) {
            x = res;
        } else if (ci.kind == KIND_TARGET_SOLVED) {
            const int16_t *rows = ws.atomRows + (size_t)c * m;
            const int topLim = ci.ptop > 0 ? rows[ci.ptop - 1] + 1 : 0;   // pool above: rows < topLim
            const int botLim = ci.pbot > 0 ? rows[ci.bbase] : m;           // pool below: rows >= botLim
            x &= row_mask(w, 0, topLim) | row_mask(w, botLim, m);
        }
        bits[idx] = x & res;
    }
    __syncthreads();
    if (s_bad) {
        if (tid == 0) { I->status = RR_INFEASIBLE; I->n_moves = 0; }
        return;
    }

    const long long colTotal = s_base;
    long long done = 0;          // moves of the receiver units so far
    long long steps = 0;
    for (int j = c0; j < c1; ++j) {
        const ColInfo Rj = ws.col[j];
        if (Rj.kind != KIND_RECEIVER) continue;
        const int M = Rj.nband, need = h - M, nh = h - M;
        const int16_t *hr = ws.holeRows + (size_t)(j - c0) * h;
        if (wid < 2) {
            const int got = bird_walk(bits, W, m, n, r0, r1, j, wid == 0, need, wid == 0 ? topTok : botTok);
            if (lane == 0) { if (wid == 0) s_nt = got; else s_nb = got; }
        }
        __syncthreads();
        if (wid == 0) {
            const int nt = s_nt, nb = s_nb;
            int a = -1;
            if (nt + nb >= need) {
                const int lo = max(0, need - nb), hi = min(need, nt);
                // d cost / da: one more token from above (the a-th nearest)
                // and one fewer from below (the (need-a+1)-th nearest)
                a = split_search(lo, hi, [&](int aa) {
                    const int tv = topTok[aa - 1], bv = botTok[need - aa];
                    const int tpos = tok_row(tv) - iabs(tok_col(tv) - j);
                    const int bpos = tok_row(bv) + iabs(tok_col(bv) - j);
                    return (r0 + aa - 1 - tpos) + (2 * band_P(hr, nh, M, r0, r0 + aa - 1) - M) +
                           (r0 + h - need + aa - 1 - bpos);
                });
            }
            if (lane == 0) s_a = a;
        }
        __syncthreads();
        const int a = s_a;
        if (a < 0) {             // cannot happen when the total surplus is >= 0
            if (tid == 0) set_status(I, RR_ERR_INTERNAL);
            return;
        }
        // Targets r0 + k: k < a from above (nearest deepest), then the band
        // atoms in order, then from below (nearest shallowest). Emission as
        // every unit: toward larger rows deepest first, then toward smaller
        // rows shallowest first; isolated band atoms are dropped.
        const int kd_end = a + band_P(hr, nh, M, r0, r0 + a - 1);
        const int ku_start = a + band_P(hr, nh, M, r0, r0 + a);
        const int16_t *own = ws.atomRows + (size_t)j * m;
        const long long base = colTotal + done;
        for (int k = tid; k < h; k += blockDim.x) {
            int row, col;
            if (k < a) { const int v = topTok[a - 1 - k]; row = tok_row(v); col = tok_col(v); }
            else if (k < a + M) { row = own[Rj.ntop + (k - a)]; col = j; }
            else { const int v = botTok[k - a - M]; row = tok_row(v); col = tok_col(v); }
            int pos;
            if (k < kd_end) pos = kd_end - 1 - k;
            else if (k >= ku_start) pos = kd_end + (k - ku_start);
            else continue;
            const long long o = base + pos;
            if (o < I->cap_moves) I->moves[o] = rr_move{row, col, r0 + k, j};
            steps += iabs(r0 + k - row) + iabs(j - col);
        }
        // the chosen tokens leave the reservoirs
        for (int l = tid; l < need; l += blockDim.x) {
            const int v = l < a ? topTok[l] : botTok[l - a];
            const int row = tok_row(v), col = tok_col(v);
            atomicAnd(&bits[(size_t)col * W + (row >> 5)], ~(1u << (row & 31)));
        }
        done += kd_end + (h - ku_start);
        __syncthreads();
    }
    add_steps(I, steps);
    if (tid == 0) {
        const long long total = colTotal + done;
        I->n_moves = total;
        if (total > I->cap_moves) set_status(I, RR_ERR_CAPACITY);
    }
}

} // namespace rrk
