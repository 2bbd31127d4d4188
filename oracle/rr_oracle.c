/*
 * rr_oracle.c -- sequential CPU oracle for the improved red-rec planner
 * (Alg. 1, Sec. III.C, in the column order of the parallel variant of
 * Sec. III.D), the bird planner (Alg. 2, Sec. III.E) and the batching
 * routine (Alg. 4 with the local constraint set of Sec. IV), arXiv
 * 2504.06182.
 *
 * TEST INFRASTRUCTURE ONLY: the plain, slow statement of what the planner
 * computes. The tests, the smoke check and the benchmark's CPU baselines
 * (its cpu_baseline legs and its reference arm) are its only users; it
 * shares no code with the CUDA library.
 *
 * Every choice the paper leaves open is fixed here, once:
 *  - Exact 1D with a contiguous target interval (Sec. III.A, "Assignment"):
 *    a distance-minimising T-saturating matching on a path matches targets,
 *    in order, to a contiguous window of the sorted sources; every window is
 *    evaluated and the smallest window start wins ties.
 *  - Target sub-rectangles (the paper only treats a full-width band and says
 *    the general case is an adaptation whose details it omits, Sec. III.C):
 *    a column outside the target columns is solved in the column phase with
 *    its own reservoir cells as virtual targets, so that its band-row atoms
 *    are pushed out into its reservoir rows where they can be donated. With
 *    a full-width target there are no such columns and the method is the
 *    paper's. The strict reading (mode `strict`) leaves every outer column
 *    as it is: only its reservoir-row atoms are donatable, as the paper's
 *    donors donate only reservoir atoms, and its band-row atoms never move.
 *  - Emission order inside one solve unit (Sec. III.A, "Generating moves"):
 *    paths that move toward larger row indices first, by descending target
 *    row, then paths toward smaller row indices by ascending target row, so
 *    that the path farthest along its direction runs first; isolated paths
 *    are dropped. Units: column phase in column order, then receivers in the
 *    order they become saturated.
 *  - Pairing (Sec. III.C, the three-level rule): donor/receiver pairs whose
 *    columns in between are all at zero surplus; maximise the tokens
 *    exchanged, then minimise the column gap, then the receiver's distance to
 *    saturation, then the receiver index, then the donor index.
 *  - Redistribution as a 1D instance (Sec. III.C): a receiver is solved once,
 *    when saturated, from its own atoms, the atoms delayed for it, and x
 *    atoms of the final donor's reservoir; the x atoms are the a nearest to
 *    the target band from above and x-a nearest from below for the a of
 *    least total vertical distance (largest a on ties). Tokens projected onto
 *    one row are ordered, above the band, farthest column first (right before
 *    left at equal distance), below it nearest column first (left before
 *    right), so nearer tokens get the deeper targets and clear the shared
 *    corridor first.
 *  - bird (Sec. III.E): the column phase is red-rec's; then the unsolved
 *    columns are taken left to right. The generalised 1D instance of column
 *    j holds all of j's atoms at their rows and every atom in a reservoir row
 *    of every other column, projected along its diagonal onto j (row - d
 *    above the band, row + d below it, d the column distance). The optimal
 *    window over the sorted tokens (smallest start on ties) fixes how many
 *    tokens each vertex gives; a vertex holding several gives its nearest
 *    columns' tokens, left before right at equal distance. Tokens are then
 *    matched in order, with the same order on one vertex as red-rec's
 *    projected tokens (nearer tokens get the targets farther along their
 *    direction), and emitted as one unit.
 *  - Dependencies Gamma (Sec. IV, "Input to the batching routine"): path b
 *    depends on every earlier path whose vertex set meets its own.
 *  - Batching (Alg. 4 + Sec. IV "Constrained batching"): ready paths are
 *    visited in ascending id; a path's next step joins the batch iff it moves
 *    in the first member's direction and its current cell shares a row or a
 *    column with the current cell of every member already in the batch.
 */
#include "rr_oracle.h"

#include <stdlib.h>
#include <string.h>

enum { OK = 0, INFEASIBLE = 1, E_ARG = -1, E_CAP = -2, E_NOMEM = -5, E_BUG = -6 };

typedef struct { int32_t sr, sc, dr, dc; } mv_t;
typedef struct { mv_t *v; int64_t n, cap; int err; } mvvec_t;
typedef struct { int32_t row, col; } tok_t;

static void mv_push(mvvec_t *L, mv_t x)
{
    if (L->err) return;
    if (L->n == L->cap) {
        int64_t nc = L->cap ? 2 * L->cap : 256;
        mv_t *p = (mv_t *)realloc(L->v, (size_t)nc * sizeof(mv_t));
        if (!p) { L->err = 1; return; }
        L->v = p; L->cap = nc;
    }
    L->v[L->n++] = x;
}

static int cmp_i32_asc(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}
static int cmp_i32_desc(const void *a, const void *b) { return cmp_i32_asc(b, a); }
static int cmp_mv_dr(const void *a, const void *b)
{
    int32_t x = ((const mv_t *)a)->dr, y = ((const mv_t *)b)->dr;
    return (x > y) - (x < y);
}
static int64_t iabs64(int64_t v) { return v < 0 ? -v : v; }

/* ---------------------------------------------------------------- 1D parts */

/* Cost of matching the window s[w .. w+h) to rows r0 .. r0+h-1 in order. */
static int64_t window_cost(const int32_t *s, int w, int r0, int h)
{
    int64_t c = 0;
    for (int k = 0; k < h; ++k) c += iabs64((int64_t)s[w + k] - (r0 + k));
    return c;
}

int rro_window(const int32_t *s, int K, int r0, int h)
{
    if (!s || h < 0 || K < h) return -1;
    int best = 0;
    int64_t bc = window_cost(s, 0, r0, h);
    for (int w = 1; w + h <= K; ++w) {
        int64_t c = window_cost(s, w, r0, h);
        if (c < bc) { bc = c; best = w; }
    }
    return best;
}

/* Sort rows[0..h) ascending and return sum_k |rows[k] - (r0+k)|. */
static int64_t sorted_cost(int32_t *rows, int h, int r0)
{
    qsort(rows, (size_t)h, sizeof(int32_t), cmp_i32_asc);
    int64_t c = 0;
    for (int k = 0; k < h; ++k) c += iabs64((int64_t)rows[k] - (r0 + k));
    return c;
}

int rro_split(const int32_t *mand, int nm, const int32_t *top, int nt,
              const int32_t *bot, int nb, int x, int r0, int h,
              int64_t *cost_out)
{
    if (nm < 0 || nt < 0 || nb < 0 || x < 0 || x > nt + nb || nm + x != h) return -1;
    int32_t *t = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nt + 1));
    int32_t *b = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nb + 1));
    int32_t *rows = (int32_t *)malloc(sizeof(int32_t) * (size_t)(h + 1));
    if (!t || !b || !rows) { free(t); free(b); free(rows); return -1; }
    if (nt) memcpy(t, top, sizeof(int32_t) * (size_t)nt);
    if (nb) memcpy(b, bot, sizeof(int32_t) * (size_t)nb);
    qsort(t, (size_t)nt, sizeof(int32_t), cmp_i32_desc);   /* nearest the band first */
    qsort(b, (size_t)nb, sizeof(int32_t), cmp_i32_asc);    /* nearest the band first */
    int lo = x - nb > 0 ? x - nb : 0;
    int hi = x < nt ? x : nt;
    int best = -1;
    int64_t bc = 0;
    for (int a = lo; a <= hi; ++a) {
        int k = 0;
        for (int i = 0; i < nm; ++i) rows[k++] = mand[i];
        for (int i = 0; i < a; ++i) rows[k++] = t[i];
        for (int i = 0; i < x - a; ++i) rows[k++] = b[i];
        int64_t c = sorted_cost(rows, h, r0);
        if (best < 0 || c <= bc) { bc = c; best = a; }     /* largest a on ties */
    }
    if (cost_out) *cost_out = bc;
    free(t); free(b); free(rows);
    return best;
}

/* Emit one solve unit: every path of the unit ends in one column at distinct
 * rows. Paths toward larger rows run first, deepest target first; then paths
 * toward smaller rows, shallowest target first; isolated paths are dropped. */
static int emit_unit(mvvec_t *out, mv_t *u, int cnt)
{
    qsort(u, (size_t)cnt, sizeof(mv_t), cmp_mv_dr);
    for (int k = 1; k < cnt; ++k)
        if (u[k].dr == u[k - 1].dr || u[k].dc != u[0].dc) return E_BUG;
    for (int k = cnt - 1; k >= 0; --k)
        if (u[k].dr > u[k].sr) mv_push(out, u[k]);
    for (int k = 0; k < cnt; ++k)
        if (u[k].dr < u[k].sr) mv_push(out, u[k]);
    for (int k = 0; k < cnt; ++k)
        if (u[k].dr == u[k].sr && u[k].dc != u[k].sc) return E_BUG;
    return out->err ? E_NOMEM : OK;
}

/* ------------------------------------------------------------ the planner */

typedef struct {
    int32_t *row;      /* pool rows of this column (its reservoir atoms) */
    uint8_t *live;     /* still in the pool */
    int cnt;
} pool_t;

typedef struct { tok_t *v; int n, cap; } tokvec_t;

static int tok_push(tokvec_t *T, tok_t t)
{
    if (T->n == T->cap) {
        int nc = T->cap ? 2 * T->cap : 16;
        tok_t *p = (tok_t *)realloc(T->v, (size_t)nc * sizeof(tok_t));
        if (!p) return E_NOMEM;
        T->v = p; T->cap = nc;
    }
    T->v[T->n++] = t;
    return OK;
}

/* Order of tokens projected onto receiver column g_rcv (see header). The
 * comparator's parameters are thread-local so that concurrent calls (the CPU
 * baseline runs the oracle on several host threads) do not interfere. */
static _Thread_local int g_r0, g_r1, g_rcv, g_tie_bug;
static int cmp_tok(const void *pa, const void *pb)
{
    const tok_t *a = (const tok_t *)pa, *b = (const tok_t *)pb;
    if (a->row != b->row) return a->row < b->row ? -1 : 1;
    if (a->row >= g_r0 && a->row < g_r1) { g_tie_bug = 1; return 0; }
    int da = abs(a->col - g_rcv), db = abs(b->col - g_rcv);
    int ra = a->col > g_rcv, rb = b->col > g_rcv;      /* right side */
    if (a->row < g_r0) {                               /* above the band */
        if (da != db) return da > db ? -1 : 1;
        if (ra != rb) return ra ? -1 : 1;
    } else {                                           /* below the band */
        if (da != db) return da < db ? -1 : 1;
        if (ra != rb) return ra ? 1 : -1;
    }
    g_tie_bug = 1;                                     /* same cell twice */
    return 0;
}

static int sgn(int v) { return (v > 0) - (v < 0); }

int rro_plan(const uint8_t *grid, int m, int n, int r0, int c0, int r1, int c1,
             int32_t *moves, int64_t cap, int64_t *n_moves,
             int32_t *sigma_out, int32_t *events, int64_t cap_ev,
             int64_t *n_events)
{
    return rro_plan_mode(grid, m, n, r0, c0, r1, c1, moves, cap, n_moves, sigma_out, events, cap_ev,
                         n_events, 0);
}

int rro_plan_mode(const uint8_t *grid, int m, int n, int r0, int c0, int r1, int c1,
                  int32_t *moves, int64_t cap, int64_t *n_moves,
                  int32_t *sigma_out, int32_t *events, int64_t cap_ev,
                  int64_t *n_events, int strict)
{
    if (!grid || !n_moves || m < 1 || n < 1 || r0 < 0 || r0 >= r1 || r1 > m ||
        c0 < 0 || c0 >= c1 || c1 > n || cap < 0 || (cap > 0 && !moves))
        return E_ARG;
    const int h = r1 - r0, R = m - h;
    int st = OK;
    int64_t nev = 0;
    mvvec_t out = {0};
    int *K = (int *)calloc((size_t)n, sizeof(int));
    int *sigma = (int *)calloc((size_t)n, sizeof(int));
    int32_t **atoms = (int32_t **)calloc((size_t)n, sizeof(int32_t *));
    pool_t *pool = (pool_t *)calloc((size_t)n, sizeof(pool_t));
    tokvec_t *marked = (tokvec_t *)calloc((size_t)n, sizeof(tokvec_t));
    mv_t *unit = (mv_t *)malloc(sizeof(mv_t) * (size_t)(m + 1));
    tok_t *src = (tok_t *)malloc(sizeof(tok_t) * (size_t)(m + 1));
    int32_t *scratch = (int32_t *)malloc(sizeof(int32_t) * (size_t)(3 * m + 3));
    if (!K || !sigma || !atoms || !pool || !marked || !unit || !src || !scratch) { st = E_NOMEM; goto done; }

    /* Atom rows of every column, top to bottom. */
    for (int c = 0; c < n; ++c) {
        for (int r = 0; r < m; ++r) K[c] += grid[(size_t)r * n + c] != 0;
        atoms[c] = (int32_t *)malloc(sizeof(int32_t) * (size_t)(K[c] + 1));
        pool[c].row = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m + 1));
        pool[c].live = (uint8_t *)calloc((size_t)(m + 1), 1);
        if (!atoms[c] || !pool[c].row || !pool[c].live) { st = E_NOMEM; goto done; }
        int k = 0;
        for (int r = 0; r < m; ++r)
            if (grid[(size_t)r * n + c]) atoms[c][k++] = r;
    }

    /* Column phase (Alg. 1 first loop; Sec. III.D solves every column of
     * non-negative surplus at the outset). Surplus sigma_i = |S n C_i| - |T n C_i|. */
    for (int c = 0; c < n; ++c) {
        const int32_t *s = atoms[c];
        int cnt = 0;
        pool[c].cnt = 0;
        if (c >= c0 && c < c1) {
            sigma[c] = K[c] - h;
            if (sigma[c] < 0) continue;                  /* receiver: waits for donors */
            int w = rro_window(s, K[c], r0, h);
            if (w < 0) { st = E_BUG; goto done; }
            for (int k = 0; k < h; ++k) unit[cnt++] = (mv_t){s[w + k], c, r0 + k, c};
            for (int k = 0; k < K[c]; ++k) {
                if (k >= w && k < w + h) continue;
                if (s[k] >= r0 && s[k] < r1) { st = E_BUG; goto done; }   /* excess lies in the reservoir */
                pool[c].row[pool[c].cnt] = s[k];
                pool[c].live[pool[c].cnt++] = 1;
            }
        } else if (!strict && K[c] >= R) {
            /* Virtual targets = the reservoir cells 0..r0-1 and r1..m-1. */
            const int nbot = m - r1;
            for (int k = 0; k < r0; ++k) unit[cnt++] = (mv_t){s[k], c, k, c};
            for (int k = 0; k < nbot; ++k) unit[cnt++] = (mv_t){s[K[c] - nbot + k], c, r1 + k, c};
            for (int r = 0; r < m; ++r) {
                if (r >= r0 && r < r1) continue;
                pool[c].row[pool[c].cnt] = r;
                pool[c].live[pool[c].cnt++] = 1;
            }
            sigma[c] = R;
        } else {
            for (int k = 0; k < K[c]; ++k) {
                if (s[k] >= r0 && s[k] < r1) continue;
                pool[c].row[pool[c].cnt] = s[k];
                pool[c].live[pool[c].cnt++] = 1;
            }
            sigma[c] = pool[c].cnt;
        }
        if ((st = emit_unit(&out, unit, cnt)) != OK) goto done;
    }
    if (sigma_out) memcpy(sigma_out, sigma, sizeof(int) * (size_t)n);

    /* Every column must be saturable: total surplus must be non-negative. */
    {
        int64_t tot = 0;
        for (int c = 0; c < n; ++c) tot += sigma[c];
        if (tot < 0) { st = INFEASIBLE; out.n = 0; goto done; }
    }

    /* Main loop of Alg. 1. */
    for (int iter = 0;; ++iter) {
        int any_neg = 0;
        for (int c = 0; c < n; ++c) any_neg |= sigma[c] < 0;
        if (!any_neg) break;
        if (iter > n) { st = E_BUG; goto done; }

        /* Best donor-receiver pair: adjacent in the sequence of columns with
         * non-zero surplus (all columns strictly between are at zero). */
        int bi = -1, bj = -1, bx = 0, bd = 0, bneed = 0;
        int prev = -1;
        for (int c = 0; c < n; ++c) {
            if (sigma[c] == 0) continue;
            if (prev >= 0 && sgn(sigma[prev]) != sgn(sigma[c])) {
                int i = sigma[prev] > 0 ? prev : c;
                int j = sigma[prev] > 0 ? c : prev;
                int need = -sigma[j];
                int x = sigma[i] < need ? sigma[i] : need;
                int d = abs(i - j);
                int better;
                if (bi < 0) better = 1;
                else if (x != bx) better = x > bx;
                else if (d != bd) better = d < bd;
                else if (need != bneed) better = need < bneed;
                else if (j != bj) better = j < bj;
                else better = i < bi;
                if (better) { bi = i; bj = j; bx = x; bd = d; bneed = need; }
            }
            prev = c;
        }
        if (bi < 0) { st = E_BUG; goto done; }
        const int i = bi, j = bj, x = bx;
        int kase = sigma[i] > -sigma[j] ? 1 : (sigma[i] == -sigma[j] ? 2 : 3);
        int a_rec = 0;

        if (kase == 3) {
            /* Donor exhausted: all its remaining atoms are marked for j. */
            for (int k = 0; k < pool[i].cnt; ++k) {
                if (!pool[i].live[k]) continue;
                if (pool[i].row[k] < r0) ++a_rec;
                if (tok_push(&marked[j], (tok_t){pool[i].row[k], i}) != OK) { st = E_NOMEM; goto done; }
                pool[i].live[k] = 0;
            }
            sigma[j] += sigma[i];
            sigma[i] = 0;
        } else {
            /* Receiver saturated now: build and solve its 1D instance. */
            int nlive = 0;
            for (int k = 0; k < pool[i].cnt; ++k) nlive += pool[i].live[k];
            if (K[j] + marked[j].n + x != h || x > nlive || (kase == 2 && nlive != x)) { st = E_BUG; goto done; }
            int ns = 0;
            for (int k = 0; k < K[j]; ++k) src[ns++] = (tok_t){atoms[j][k], j};
            for (int k = 0; k < marked[j].n; ++k) src[ns++] = marked[j].v[k];
            if (kase == 2) {
                for (int k = 0; k < pool[i].cnt; ++k) {
                    if (!pool[i].live[k]) continue;
                    if (pool[i].row[k] < r0) ++a_rec;
                    src[ns++] = (tok_t){pool[i].row[k], i};
                    pool[i].live[k] = 0;
                }
            } else {
                int32_t *mand = scratch, *top = scratch + m + 1, *bot = scratch + 2 * m + 2;
                int nt = 0, nb = 0;
                for (int k = 0; k < ns; ++k) mand[k] = src[k].row;
                for (int k = 0; k < pool[i].cnt; ++k) {
                    if (!pool[i].live[k]) continue;
                    if (pool[i].row[k] < r0) top[nt++] = pool[i].row[k];
                    else bot[nb++] = pool[i].row[k];
                }
                int a = rro_split(mand, ns, top, nt, bot, nb, x, r0, h, NULL);
                if (a < 0) { st = E_BUG; goto done; }
                a_rec = a;
                /* rro_split sorted nothing in place: pick the a nearest top
                 * rows and x-a nearest bottom rows of the live pool. */
                qsort(top, (size_t)nt, sizeof(int32_t), cmp_i32_desc);
                qsort(bot, (size_t)nb, sizeof(int32_t), cmp_i32_asc);
                int tlim = a > 0 ? top[a - 1] : r0;          /* take top rows >= tlim */
                int blim = x - a > 0 ? bot[x - a - 1] : r1 - 1; /* take bottom rows <= blim */
                for (int k = 0; k < pool[i].cnt; ++k) {
                    if (!pool[i].live[k]) continue;
                    int r = pool[i].row[k];
                    if ((r < r0 && r >= tlim) || (r >= r1 && r <= blim)) {
                        src[ns++] = (tok_t){r, i};
                        pool[i].live[k] = 0;
                    }
                }
            }
            if (ns != h) { st = E_BUG; goto done; }
            g_r0 = r0; g_r1 = r1; g_rcv = j; g_tie_bug = 0;
            qsort(src, (size_t)ns, sizeof(tok_t), cmp_tok);
            if (g_tie_bug) { st = E_BUG; goto done; }
            for (int k = 0; k < h; ++k) unit[k] = (mv_t){src[k].row, src[k].col, r0 + k, j};
            if ((st = emit_unit(&out, unit, h)) != OK) goto done;
            sigma[i] -= x;
            sigma[j] = 0;
        }
        if (events && nev < cap_ev) {
            int32_t *e = events + 5 * nev;
            e[0] = kase; e[1] = i; e[2] = j; e[3] = x; e[4] = a_rec;
        }
        ++nev;
    }

done:
    if (st == OK || st == INFEASIBLE) {
        if (out.err) st = E_NOMEM;
    }
    if (st == OK || st == INFEASIBLE) {
        *n_moves = out.n;
        if (out.n > cap) st = E_CAP;
        else if (out.n) memcpy(moves, out.v, sizeof(mv_t) * (size_t)out.n);
    }
    if (n_events) *n_events = nev;
    if (atoms) for (int c = 0; c < n; ++c) free(atoms[c]);
    if (pool) for (int c = 0; c < n; ++c) { free(pool[c].row); free(pool[c].live); }
    if (marked) for (int c = 0; c < n; ++c) free(marked[c].v);
    free(K); free(sigma); free(atoms); free(pool); free(marked);
    free(unit); free(src); free(scratch); free(out.v);
    return st;
}

/* -------------------------------------------------------- the bird planner */

/* One token of the generalised 1D instance of a receiver column (Sec. III.E).
 * pos is the token's vertex on the receiver's column: its own row for the
 * receiver's own atoms; for an atom in a reservoir row v of another column at
 * column distance d, v - d above the band and v + d below it, so that
 * |pos - t| is the Manhattan distance to band trap t of the receiver. */
typedef struct { int32_t pos, row, col; } btok_t;

/* Order of the tokens of receiver g_rcv: by vertex; on one vertex above the
 * band the farther column first (right before left at equal distance), below
 * it the nearer column first (left before right). The nearest tokens of a
 * vertex are thus the last ones above the band and the first ones below it. */
static int cmp_btok(const void *pa, const void *pb)
{
    const btok_t *a = (const btok_t *)pa, *b = (const btok_t *)pb;
    if (a->pos != b->pos) return a->pos < b->pos ? -1 : 1;
    int da = abs(a->col - g_rcv), db = abs(b->col - g_rcv);
    int ra = a->col > g_rcv, rb = b->col > g_rcv;
    if (a->pos < g_r0) {
        if (da != db) return da > db ? -1 : 1;
        if (ra != rb) return ra ? -1 : 1;
    } else {
        if (da != db) return da < db ? -1 : 1;
        if (ra != rb) return ra ? 1 : -1;
    }
    g_tie_bug = 1;                     /* same cell twice */
    return 0;
}

/* Executes one unit on the occupancy grid: every source is vacated, then
 * every destination filled (an isolated path leaves its atom in place). */
static void apply_unit(uint8_t *cur, int n, const mv_t *u, int cnt)
{
    for (int k = 0; k < cnt; ++k) cur[(size_t)u[k].sr * n + u[k].sc] = 0;
    for (int k = 0; k < cnt; ++k) cur[(size_t)u[k].dr * n + u[k].dc] = 1;
}

static int bird_impl(const uint8_t *grid, int m, int n, int r0, int c0, int r1, int c1,
                     int32_t *moves, int64_t cap, int64_t *n_moves,
                     int32_t *units, int64_t cap_units, int64_t *n_units, int strict,
                     int64_t max_units);

int rro_bird(const uint8_t *grid, int m, int n, int r0, int c0, int r1, int c1,
             int32_t *moves, int64_t cap, int64_t *n_moves,
             int32_t *units, int64_t cap_units, int64_t *n_units)
{
    return bird_impl(grid, m, n, r0, c0, r1, c1, moves, cap, n_moves, units, cap_units, n_units, 0, -1);
}

int rro_bird_mode(const uint8_t *grid, int m, int n, int r0, int c0, int r1, int c1,
                  int32_t *moves, int64_t cap, int64_t *n_moves,
                  int32_t *units, int64_t cap_units, int64_t *n_units, int strict)
{
    return bird_impl(grid, m, n, r0, c0, r1, c1, moves, cap, n_moves, units, cap_units, n_units, strict, -1);
}

int rro_bird_prefix(const uint8_t *grid, int m, int n, int r0, int c0, int r1, int c1,
                    int32_t *moves, int64_t cap, int64_t *n_moves, int64_t max_units)
{
    if (max_units < 0) return E_ARG;
    return bird_impl(grid, m, n, r0, c0, r1, c1, moves, cap, n_moves, NULL, 0, NULL, 0, max_units);
}

static int bird_impl(const uint8_t *grid, int m, int n, int r0, int c0, int r1, int c1,
                     int32_t *moves, int64_t cap, int64_t *n_moves,
                     int32_t *units, int64_t cap_units, int64_t *n_units, int strict,
                     int64_t max_units)
{
    if (!grid || !n_moves || m < 1 || n < 1 || r0 < 0 || r0 >= r1 || r1 > m ||
        c0 < 0 || c0 >= c1 || c1 > n || cap < 0 || (cap > 0 && !moves))
        return E_ARG;
    const int h = r1 - r0, R = m - h;
    int st = OK;
    int64_t nu = 0, tot = 0;
    mvvec_t out = {0};
    uint8_t *cur = (uint8_t *)malloc((size_t)m * n);
    uint8_t *recv = (uint8_t *)calloc((size_t)n, 1);
    int32_t *rows = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m + 1));
    mv_t *unit = (mv_t *)malloc(sizeof(mv_t) * (size_t)(m + 1));
    btok_t *T = (btok_t *)malloc(sizeof(btok_t) * ((size_t)m * n + 1));
    int32_t *pos = (int32_t *)malloc(sizeof(int32_t) * ((size_t)m * n + 1));
    uint8_t *take = (uint8_t *)malloc((size_t)m * n + 1);
    if (!cur || !recv || !rows || !unit || !T || !pos || !take) { st = E_NOMEM; goto done; }
    memcpy(cur, grid, (size_t)m * n);
    for (size_t v = 0; v < (size_t)m * n; ++v) cur[v] = grid[v] != 0;

    /* Columns of non-negative surplus are solved first with the exact 1D
     * algorithm, exactly as in red-rec's column phase (including the
     * virtual solve of columns outside the target columns). */
    for (int c = 0; c < n; ++c) {
        int K = 0, cnt = 0;
        for (int r = 0; r < m; ++r) if (cur[(size_t)r * n + c]) rows[K++] = r;
        if (c >= c0 && c < c1) {
            tot += K - h;
            if (K < h) { recv[c] = 1; continue; }
            int w = rro_window(rows, K, r0, h);
            if (w < 0) { st = E_BUG; goto done; }
            for (int k = 0; k < h; ++k) unit[cnt++] = (mv_t){rows[w + k], c, r0 + k, c};
        } else if (!strict && K >= R) {
            const int nbot = m - r1;
            for (int k = 0; k < r0; ++k) unit[cnt++] = (mv_t){rows[k], c, k, c};
            for (int k = 0; k < nbot; ++k) unit[cnt++] = (mv_t){rows[K - nbot + k], c, r1 + k, c};
            tot += R;
        } else {
            for (int k = 0; k < K; ++k) tot += rows[k] < r0 || rows[k] >= r1;
        }
        apply_unit(cur, n, unit, cnt);
        if ((st = emit_unit(&out, unit, cnt)) != OK) goto done;
    }
    if (tot < 0) { st = INFEASIBLE; out.n = 0; goto done; }

    /* Main loop of the bird algorithm: the leftmost unsolved column is filled
     * from every token of the grid at once, through its generalised 1D
     * instance; then the next one. */
    for (int j = c0; j < c1; ++j) {
        if (!recv[j]) continue;
        if (max_units >= 0 && nu >= max_units) break;
        int nt = 0;
        for (int c = 0; c < n; ++c)
            for (int r = 0; r < m; ++r) {
                if (!cur[(size_t)r * n + c]) continue;
                const int d = abs(c - j);
                if (c == j) T[nt++] = (btok_t){r, r, c};
                else if (r < r0) T[nt++] = (btok_t){r - d, r, c};
                else if (r >= r1) T[nt++] = (btok_t){r + d, r, c};
            }
        if (nt < h) { st = E_BUG; goto done; }
        g_r0 = r0; g_r1 = r1; g_rcv = j; g_tie_bug = 0;
        qsort(T, (size_t)nt, sizeof(btok_t), cmp_btok);
        if (g_tie_bug) { st = E_BUG; goto done; }
        for (int k = 0; k < nt; ++k) pos[k] = T[k].pos;
        /* Generalised exact 1D: the optimal window gives how many tokens each
         * vertex gives; a vertex holding several gives its nearest ones. */
        const int w = rro_window(pos, nt, r0, h);
        if (w < 0) { st = E_BUG; goto done; }
        memset(take, 0, (size_t)nt);
        int ntop = 0, nbot = 0;
        for (int k = w; k < w + h;) {
            int e = k;
            while (e < w + h && pos[e] == pos[k]) ++e;     /* window part on this vertex */
            int g0 = k, g1 = e;                            /* all tokens on this vertex */
            while (g0 > 0 && pos[g0 - 1] == pos[k]) --g0;
            while (g1 < nt && pos[g1] == pos[k]) ++g1;
            const int want = e - k;
            if (pos[k] < r0) for (int q = g1 - want; q < g1; ++q) take[q] = 1;
            else for (int q = g0; q < g0 + want; ++q) take[q] = 1;
            if (pos[k] < r0) ntop += want;
            else if (pos[k] >= r1) nbot += want;
            k = e;
        }
        int cnt = 0;
        for (int k = 0; k < nt; ++k)
            if (take[k]) { unit[cnt] = (mv_t){T[k].row, T[k].col, r0 + cnt, j}; ++cnt; }
        if (cnt != h) { st = E_BUG; goto done; }
        apply_unit(cur, n, unit, cnt);
        if ((st = emit_unit(&out, unit, cnt)) != OK) goto done;
        if (units && nu < cap_units) {
            units[3 * nu] = j; units[3 * nu + 1] = ntop; units[3 * nu + 2] = nbot;
        }
        ++nu;
    }

done:
    if (st == OK || st == INFEASIBLE) {
        if (out.err) st = E_NOMEM;
    }
    if (st == OK || st == INFEASIBLE) {
        *n_moves = out.n;
        if (out.n > cap) st = E_CAP;
        else if (out.n) memcpy(moves, out.v, sizeof(mv_t) * (size_t)out.n);
    }
    if (n_units) *n_units = nu;
    free(cur); free(recv); free(rows); free(unit); free(T); free(pos); free(take); free(out.v);
    return st;
}

/* ------------------------------------------------------- batching routine */

/* Cell visited after t elementary steps of move p (row first, then column). */
static void path_cell(const mv_t *p, int t, int *r, int *c)
{
    int hl = abs(p->dc - p->sc);
    if (t <= hl) { *r = p->sr; *c = p->sc + t * sgn(p->dc - p->sc); }
    else { *r = p->sr + (t - hl) * sgn(p->dr - p->sr); *c = p->dc; }
}
static int path_dir(const mv_t *p, int t)
{
    int hl = abs(p->dc - p->sc);
    if (t < hl) return p->dc > p->sc ? 3 : 2;
    return p->dr > p->sr ? 1 : 0;
}

static int batch_impl(const int32_t *moves_in, int64_t n_moves, int m, int n,
                      int64_t max_ops, int32_t *ops, int64_t cap_ops, int32_t *members,
                      int64_t cap_members, int64_t *n_ops, int64_t *n_members);

int rro_batch(const int32_t *moves_in, int64_t n_moves, int m, int n,
              int32_t *ops, int64_t cap_ops, int32_t *members,
              int64_t cap_members, int64_t *n_ops, int64_t *n_members)
{
    return batch_impl(moves_in, n_moves, m, n, -1, ops, cap_ops, members, cap_members, n_ops, n_members);
}

int rro_batch_prefix(const int32_t *moves_in, int64_t n_moves, int m, int n, int64_t max_ops,
                     int32_t *ops, int64_t cap_ops, int32_t *members,
                     int64_t cap_members, int64_t *n_ops, int64_t *n_members)
{
    if (max_ops < 0) return E_ARG;
    return batch_impl(moves_in, n_moves, m, n, max_ops, ops, cap_ops, members, cap_members, n_ops, n_members);
}

static int batch_impl(const int32_t *moves_in, int64_t n_moves, int m, int n,
                      int64_t max_ops, int32_t *ops, int64_t cap_ops, int32_t *members,
                      int64_t cap_members, int64_t *n_ops, int64_t *n_members)
{
    if (!n_ops || !n_members || m < 1 || n < 1 || n_moves < 0 || (n_moves > 0 && !moves_in))
        return E_ARG;
    const mv_t *P = (const mv_t *)moves_in;
    const int64_t k = n_moves;
    const int64_t ncell = (int64_t)m * n;
    int st = OK;
    int *len = (int *)malloc(sizeof(int) * (size_t)(k + 1));
    int *prog = (int *)calloc((size_t)(k + 1), sizeof(int));
    int64_t *blocked = (int64_t *)calloc((size_t)(k + 1), sizeof(int64_t));
    int64_t *off = (int64_t *)calloc((size_t)(ncell + 1), sizeof(int64_t));
    int64_t *head = (int64_t *)calloc((size_t)(ncell + 1), sizeof(int64_t));
    int32_t *cover = NULL;
    int32_t *ready = (int32_t *)malloc(sizeof(int32_t) * (size_t)(k + 1));
    int32_t *Q = (int32_t *)malloc(sizeof(int32_t) * (size_t)(k + 1));
    int32_t *acc = (int32_t *)malloc(sizeof(int32_t) * (size_t)(k + 1));
    int32_t *accr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(k + 1));
    int32_t *accc = (int32_t *)malloc(sizeof(int32_t) * (size_t)(k + 1));
    int32_t *newly = (int32_t *)malloc(sizeof(int32_t) * (size_t)(k + 1));
    int32_t *opv = NULL, *memv = NULL;
    int64_t nop = 0, nmem = 0, opcap = 0, memcap = 0;
    int64_t nready = 0, unfinished = k;
    if (!len || !prog || !blocked || !off || !head || !ready || !Q || !acc || !accr || !accc || !newly) {
        st = E_NOMEM; goto done;
    }
    for (int64_t b = 0; b < k; ++b) {
        const mv_t *p = &P[b];
        if (p->sr < 0 || p->sr >= m || p->dr < 0 || p->dr >= m || p->sc < 0 || p->sc >= n ||
            p->dc < 0 || p->dc >= n || (p->sr == p->dr && p->sc == p->dc)) { st = E_ARG; goto done; }
        len[b] = abs(p->dc - p->sc) + abs(p->dr - p->sr);
    }
    /* Gamma: for every cell, the moves whose path covers it, in list order. */
    for (int64_t b = 0; b < k; ++b)
        for (int t = 0; t <= len[b]; ++t) {
            int r, c; path_cell(&P[b], t, &r, &c);
            off[(int64_t)r * n + c + 1]++;
        }
    for (int64_t v = 0; v < ncell; ++v) off[v + 1] += off[v];
    cover = (int32_t *)malloc(sizeof(int32_t) * (size_t)(off[ncell] + 1));
    if (!cover) { st = E_NOMEM; goto done; }
    memcpy(head, off, sizeof(int64_t) * (size_t)ncell);
    for (int64_t b = 0; b < k; ++b)
        for (int t = 0; t <= len[b]; ++t) {
            int r, c; path_cell(&P[b], t, &r, &c);
            int64_t v = (int64_t)r * n + c;
            cover[head[v]++] = (int32_t)b;
        }
    memcpy(head, off, sizeof(int64_t) * (size_t)ncell);   /* head[v]: earliest unfinished coverer */
    /* A move waits on every cell where an earlier move also passes. */
    for (int64_t b = 0; b < k; ++b) {
        for (int t = 0; t <= len[b]; ++t) {
            int r, c; path_cell(&P[b], t, &r, &c);
            int64_t v = (int64_t)r * n + c;
            if (cover[off[v]] != b) blocked[b]++;
        }
        if (blocked[b] == 0) ready[nready++] = (int32_t)b;   /* ascending ids */
    }

    while (unfinished > 0 && (max_ops < 0 || nop < max_ops)) {
        if (nready == 0) { st = E_BUG; goto done; }
        int64_t nq = nready, na = 0, nn = 0;
        memcpy(Q, ready, sizeof(int32_t) * (size_t)nq);
        int d0 = -1;
        for (int64_t q = 0; q < nq; ++q) {
            int32_t b = Q[q];
            int r, c; path_cell(&P[b], prog[b], &r, &c);
            int d = path_dir(&P[b], prog[b]);
            int ok;
            if (na == 0) { ok = 1; d0 = d; }
            else {
                ok = d == d0;
                for (int64_t a = 0; ok && a < na; ++a) ok = accr[a] == r || accc[a] == c;
            }
            if (ok) { acc[na] = b; accr[na] = r; accc[na] = c; ++na; }
        }
        /* record the batch */
        if (nop == opcap) {
            opcap = opcap ? 2 * opcap : 1024;
            int32_t *p = (int32_t *)realloc(opv, sizeof(int32_t) * 3 * (size_t)opcap);
            if (!p) { st = E_NOMEM; goto done; }
            opv = p;
        }
        if (nmem + na > memcap) {
            while (nmem + na > memcap) memcap = memcap ? 2 * memcap : 4096;
            int32_t *p = (int32_t *)realloc(memv, sizeof(int32_t) * (size_t)memcap);
            if (!p) { st = E_NOMEM; goto done; }
            memv = p;
        }
        opv[3 * nop] = d0; opv[3 * nop + 1] = (int32_t)nmem; opv[3 * nop + 2] = (int32_t)na;
        ++nop;
        for (int64_t a = 0; a < na; ++a) memv[nmem++] = acc[a];
        /* advance; retire finished paths and release their cells */
        for (int64_t a = 0; a < na; ++a) {
            int32_t b = acc[a];
            if (++prog[b] < len[b]) continue;
            --unfinished;
            int64_t w = 0;
            for (int64_t q = 0; q < nready; ++q) if (ready[q] != b) ready[w++] = ready[q];
            nready = w;
            for (int t = 0; t <= len[b]; ++t) {
                int r, c; path_cell(&P[b], t, &r, &c);
                int64_t v = (int64_t)r * n + c;
                if (cover[head[v]] != b) { st = E_BUG; goto done; }
                if (++head[v] < off[v + 1]) {
                    int32_t nx = cover[head[v]];
                    if (--blocked[nx] == 0) newly[nn++] = nx;
                }
            }
        }
        /* newly ready paths join from the next batch on (sorted merge) */
        if (nn) {
            qsort(newly, (size_t)nn, sizeof(int32_t), cmp_i32_asc);
            int64_t i1 = nready - 1, i2 = nn - 1, w = nready + nn - 1;
            while (i2 >= 0) {
                if (i1 >= 0 && ready[i1] > newly[i2]) ready[w--] = ready[i1--];
                else ready[w--] = newly[i2--];
            }
            nready += nn;
        }
    }

done:
    if (st == OK) {
        *n_ops = nop; *n_members = nmem;
        if (nop > cap_ops || nmem > cap_members || (nop && !ops) || (nmem && !members)) st = E_CAP;
        else {
            if (nop) memcpy(ops, opv, sizeof(int32_t) * 3 * (size_t)nop);
            if (nmem) memcpy(members, memv, sizeof(int32_t) * (size_t)nmem);
        }
    }
    free(len); free(prog); free(blocked); free(off); free(head); free(cover);
    free(ready); free(Q); free(acc); free(accr); free(accc); free(newly);
    free(opv); free(memv);
    return st;
}
