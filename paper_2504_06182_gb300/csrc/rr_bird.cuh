// rr_bird.cuh -- planning stage of the bird algorithm (arXiv 2504.06182,
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
#pragma once
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

// Walk order: cell g of one side is layer k = floor(sqrt(g)) (the vertex
// r0-1-k above the band, r1+k below it), index i = g - k*k in the layer:
// i = 0 is column j itself, i = 2d-1 column j-d, i = 2d column j+d, on row
// r0-1-k+d above the band or r1+k-d below it. Ascending g is the order in
// which the optimal window takes tokens (nearest vertex first, then the
// nearer column, left before right).
__device__ __forceinline__ void walk_cell(int g, int j, int r0, int r1, bool top, int *row, int *col)
{
    const int k = isqrt_floor(g);
    const int i = g - k * k;
    const int d = (i + 1) >> 1;
    *col = d == 0 ? j : ((i & 1) ? j - d : j + d);
    *row = top ? r0 - 1 - k + d : r1 + k - d;
}

// Walks cells g in [g, gEnd) in order (one warp), appending the tokens found
// to list[got ..] until `need` are held. Returns the tokens held; *gNext is
// the first cell not examined.
__device__ inline int walk_range(const uint32_t *bits, int W, int m, int n, int r0, int r1, int j, bool top, int need,
                          int g, int gEnd, int maxIter, int got, int32_t *list, int *gNext)
{
    const int lane = threadIdx.x & 31;
    for (int it = 0; got < need && g < gEnd && it < maxIter; ++it, g += 32) {
        const int gl = g + lane;
        int row, col;
        walk_cell(gl, j, r0, r1, top, &row, &col);
        bool occ = false;
        if (gl < gEnd && col >= 0 && col < n && row >= 0 && row < m && (top ? row < r0 : row >= r1))
            occ = (bits[(size_t)col * W + (row >> 5)] >> (row & 31)) & 1u;
        const unsigned bal = __ballot_sync(FULL, occ);
        const int rank = got + __popc(bal & ((1u << lane) - 1u));
        if (occ && rank < need) list[rank] = (row << 16) | col;
        got = min(need, got + __popc(bal));
    }
    *gNext = g;
    return got;
}

// Tokens of one side in layers <= K (one warp): per column, a masked popcount
// over the rows whose vertex is within K of the band.
__device__ inline int side_count(const uint32_t *bits, int W, int m, int n, int r0, int r1, int j, bool top, int K)
{
    const int lane = threadIdx.x & 31;
    int cnt = 0;
    for (int c = lane; c < n; c += 32) {
        const int d = iabs(c - j);
        if (d > K) continue;
        const int lo = top ? max(0, r0 - 1 - K + d) : r1;
        const int hi = top ? r0 : min(m, r1 + K - d + 1);
        for (int w = lo >> 5; w <= (hi - 1) >> 5; ++w) cnt += __popc(bits[(size_t)c * W + w] & row_mask(w, lo, hi));
    }
    return warp_sum(cnt);
}

// Sorts a[0..len) ascending (one warp, bitonic network over the next power
// of two; the entries past len are padding and must fit in the buffer).
__device__ inline void warp_sort_u32(uint32_t *a, int len)
{
    const int lane = threadIdx.x & 31;
    if (len <= 1) return;
    int P = 1;
    while (P < len) P <<= 1;
    for (int i = len + lane; i < P; i += 32) a[i] = 0xffffffffu;
    __syncwarp();
    for (int k = 2; k <= P; k <<= 1)
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            for (int i = lane; i < P; i += 32) {
                const int ij = i ^ jj;
                if (ij > i) {
                    const uint32_t x = a[i], y = a[ij];
                    if ((x > y) == ((i & k) == 0)) { a[i] = y; a[ij] = x; }
                }
            }
            __syncwarp();
        }
}

// Smallest layer K >= lo at which one side holds `need` tokens, kmax when it
// never does (one warp); the layers below lo hold fewer. The search starts
// from `guess` (the previous receiver's cut-off on this side: the
// reservoirs change little from one column to the next), gallops toward the
// answer, then bisects. *before gets the tokens in layers < K.
__device__ inline int find_cutoff(const uint32_t *bits, int W, int m, int n, int r0, int r1, int j, bool top, int need,
                           int lo, int kmax, int guess, int *before)
{
    int kb = lo - 1, cb = kb < 0 ? 0 : -1;   // largest layer known to hold fewer than need, its count
    const int g = min(max(guess, lo), kmax);
    int hi = kmax;
    const int cg = side_count(bits, W, m, n, r0, r1, j, top, g);
    if (cg >= need) {
        hi = g;
        for (int s = 1; hi - s >= lo; s <<= 1) {
            const int t = hi - s;
            const int ct = side_count(bits, W, m, n, r0, r1, j, top, t);
            if (ct >= need) { hi = t; continue; }
            kb = t; cb = ct; lo = t + 1;
            break;
        }
    } else {
        kb = g; cb = cg; lo = g + 1;
        for (int s = 1;; s <<= 1) {
            const int t = min(g + s, kmax);
            const int ct = side_count(bits, W, m, n, r0, r1, j, top, t);
            if (ct >= need) { hi = t; break; }
            kb = t; cb = ct; lo = t + 1;
            if (t == kmax) {                    // fewer than need in all: take them all
                *before = side_count(bits, W, m, n, r0, r1, j, top, kmax - 1);
                return kmax;
            }
        }
    }
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const int cm = side_count(bits, W, m, n, r0, r1, j, top, mid);
        if (cm >= need) hi = mid;
        else { lo = mid + 1; kb = mid; cb = cm; }
    }
    *before = lo == 0 ? 0 : (kb == lo - 1 && cb >= 0 ? cb : side_count(bits, W, m, n, r0, r1, j, top, lo - 1));
    return lo;
}

// Collects, in walk order, the `need` nearest tokens of receiver j on one
// side of the band, or all of them if fewer (one warp). While the
// reservoirs near j are full the walk finds them in a few iterations. Once
// they are depleted the walk would scan the empty area cell by cell, so the
// cut-off layer K (the first at which the count reaches need) is found by
// popcounts instead (find_cutoff); the tokens of the layers before K are
// gathered by their walk index and sorted, and layer K alone is walked.
// *sparse and *kHint carry this side's state from one receiver to the next:
// after a cut-off beyond what the bounded walk would have reached, the next
// receiver skips the walk and starts the search from this cut-off.
__device__ inline int bird_side(const uint32_t *bits, int W, int m, int n, int r0, int r1, int j, bool top, int need,
                         int32_t *list, int *s_cnt, bool *sparse, int *kHint)
{
    const int lane = threadIdx.x & 31;
    if (top ? r0 == 0 : r1 == m) return 0;
    const int dmax = max(j, n - 1 - j);
    const int kmax = top ? r0 - 1 + dmax : m - 1 - r1 + dmax;   // no cell beyond this layer
    const int gAll = (kmax + 1) * (kmax + 1);
    const int walkIter = 8 + need / 8;
    int gNext, lo = 0;
    if (!*sparse) {
        const int got = walk_range(bits, W, m, n, r0, r1, j, top, need, 0, gAll, walkIter, 0, list, &gNext);
        if (got >= need || gNext >= gAll) return got;
        lo = isqrt_floor(gNext);             // layers below the walk's last one hold fewer than need
    }
    int before;
    const int K = find_cutoff(bits, W, m, n, r0, r1, j, top, need, lo, kmax, *kHint, &before);
    *kHint = K;
    *sparse = (K + 1) * (K + 1) > 32 * walkIter;
    // gather the walk indices of the tokens in layers < K, sort, decode
    if (lane == 0) *s_cnt = 0;
    __syncwarp();
    uint32_t *keys = (uint32_t *)list;
    for (int c = lane; c < n; c += 32) {
        const int d = iabs(c - j);
        if (d > K - 1) continue;
        const int rlo = top ? max(0, r0 - 1 - (K - 1) + d) : r1;
        const int rhi = top ? r0 : min(m, r1 + (K - 1) - d + 1);
        const int i = d == 0 ? 0 : (c < j ? 2 * d - 1 : 2 * d);
        for (int w = rlo >> 5; w <= (rhi - 1) >> 5; ++w) {
            uint32_t x = bits[(size_t)c * W + w] & row_mask(w, rlo, rhi);
            while (x) {
                const int v = 32 * w + __ffs(x) - 1;
                x &= x - 1;
                const int k = (top ? r0 - 1 - v : v - r1) + d;
                const int slot = atomicAdd(s_cnt, 1);
                if (slot < before) keys[slot] = (uint32_t)(k * k + i);
            }
        }
    }
    __syncwarp();
    warp_sort_u32(keys, before);
    for (int t = lane; t < before; t += 32) {
        int row, col;
        walk_cell((int)keys[t], j, r0, r1, top, &row, &col);
        list[t] = (row << 16) | col;
    }
    __syncwarp();
    return walk_range(bits, W, m, n, r0, r1, j, top, need, K * K, (K + 1) * (K + 1), 0x7fffffff, before, list,
                      &gNext);
}

// Threads of the bird stage: two warps (one per side of the band), synchronised
// by a named barrier of their own, so that the stage also runs inside a larger
// block whose other warps wait outside it.
constexpr int BIRD_THREADS = 64;
__device__ __forceinline__ void bird_sync() { asm volatile("bar.sync 1, 64;" ::: "memory"); }

__device__ inline void s_bird(const Blk B, rr_instance *inst, JobWS *wsv, int count, int max_side)
{
    extern __shared__ uint32_t birdsm[];
    __shared__ int s_nt, s_nb, s_a, s_base, s_bad, s_nrecv, s_cnt[2];
    const int q = B.x;
    if (q >= count) return;
    rr_instance *I = &inst[q];
    if (!live(I)) return;
    JobWS &ws = wsv[q];
    const int m = I->m, n = I->n, W = (m + 31) >> 5;
    const int r0 = I->rect.r0, r1 = I->rect.r1, c0 = I->rect.c0, c1 = I->rect.c1, h = r1 - r0;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    uint32_t *bits = birdsm;                                               // n * W words
    int listCap = 1;                                                      // next power of two >= max_side
    while (listCap < max_side) listCap <<= 1;
    int32_t *topTok = (int32_t *)(birdsm + (size_t)max_side * ((max_side + 31) >> 5));
    int32_t *botTok = topTok + listCap;
    // receivers in column order (column, band atoms, atoms above the band),
    // and the current receiver's band holes and band atom rows
    int16_t *recvCol = (int16_t *)(botTok + listCap);
    int16_t *recvM = recvCol + max_side, *recvTop = recvM + max_side;
    int16_t *sHr = recvTop + max_side, *sOwn = sHr + max_side;

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
    } else if (wid == 1) {
        int nr = 0;
        for (int base = c0; base < c1; base += 32) {
            const int c = base + lane;
            bool rc = false;
            int M = 0, T = 0;
            if (c < c1) { const ColInfo ci = ws.col[c]; rc = ci.kind == KIND_RECEIVER; M = ci.nband; T = ci.ntop; }
            const unsigned bal = __ballot_sync(FULL, rc);
            if (rc) {
                const int at = nr + __popc(bal & ((1u << lane) - 1u));
                recvCol[at] = (int16_t)c; recvM[at] = (int16_t)M; recvTop[at] = (int16_t)T;
            }
            nr += __popc(bal);
        }
        if (lane == 0) s_nrecv = nr;
    }
    // Reservoir rows after the column phase: solved target columns keep the
    // atoms outside their window, outer columns with enough atoms fill every
    // reservoir trap, the others are untouched. Band rows are never read.
    for (int idx = tid; idx < n * W; idx += BIRD_THREADS) {
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
    bird_sync();
    if (s_bad) {
        if (tid == 0) { I->status = RR_INFEASIBLE; I->n_moves = 0; }
        return;
    }

    const long long colTotal = s_base;
    const int nrecv = s_nrecv;
    long long done = 0;          // moves of the receiver units so far
    long long steps = 0;
    bool sparse = false;         // this warp's side: walk skipped, search hint
    int kHint = 0;
    for (int u = 0; u < nrecv; ++u) {
        const int j = recvCol[u], M = recvM[u], ownTop = recvTop[u];
        const int need = h - M, nh = h - M;
        // this receiver's band holes and band atoms (read by the split and
        // the emission once the walks are done)
        {
            const int16_t *ghr = ws.holeRows + (size_t)(j - c0) * h;
            const int16_t *gown = ws.atomRows + (size_t)j * m + ownTop;
            for (int t = tid; t < nh; t += BIRD_THREADS) sHr[t] = ghr[t];
            for (int t = tid; t < M; t += BIRD_THREADS) sOwn[t] = gown[t];
        }
        const int16_t *hr = sHr;
        if (wid < 2) {
            const int got = bird_side(bits, W, m, n, r0, r1, j, wid == 0, need, wid == 0 ? topTok : botTok,
                                      &s_cnt[wid], &sparse, &kHint);
            if (lane == 0) { if (wid == 0) s_nt = got; else s_nb = got; }
        }
        bird_sync();
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
        bird_sync();
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
        const long long base = colTotal + done;
        for (int k = tid; k < h; k += BIRD_THREADS) {
            int row, col;
            if (k < a) { const int v = topTok[a - 1 - k]; row = tok_row(v); col = tok_col(v); }
            else if (k < a + M) { row = sOwn[k - a]; col = j; }
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
        for (int l = tid; l < need; l += BIRD_THREADS) {
            const int v = l < a ? topTok[l] : botTok[l - a];
            const int row = tok_row(v), col = tok_col(v);
            atomicAnd(&bits[(size_t)col * W + (row >> 5)], ~(1u << (row & 31)));
        }
        done += kd_end + (h - ku_start);
        bird_sync();
    }
    add_steps(I, steps);
    if (tid == 0) {
        const long long total = colTotal + done;
        I->n_moves = total;
        if (total > I->cap_moves) set_status(I, RR_ERR_CAPACITY);
    }
}

} // namespace rrk
