// rr_plan.cuh -- planning stages of the improved red-rec algorithm
// (arXiv 2504.06182, Alg. 1; Sec. III.A exact 1D, Sec. III.C redistribution,
// Sec. III.D parallel ordering: every column of non-negative surplus is
// solved up front, then the donor/receiver pairs are identified by one warp
// and the receivers are solved in parallel).
//
// Every stage takes the whole instance array; B.y selects the instance
// (B.x for the stages that run one block per instance). An instance whose
// status is not RR_OK is skipped.
#pragma once
#include "rr_internal.cuh"

namespace rrk {

// ----------------------------------------------------------------- helpers

// Row of the l-th nearest-to-band pool atom above (top) / below (bottom).
__device__ __forceinline__ int pool_top_row(const ColInfo &D, const int16_t *rows, int r0, int l)
{
    return D.kind == KIND_OUTER_FULL ? r0 - 1 - l : (int)rows[D.tbase - l];
}
__device__ __forceinline__ int pool_bot_row(const ColInfo &D, const int16_t *rows, int r1, int l)
{
    return D.kind == KIND_OUTER_FULL ? r1 + l : (int)rows[D.bbase + l];
}

// ------------------------------------------------------------ validation

__device__ inline void s_plan_setup(const Blk B, rr_instance *inst, JobWS *wsv, int count, int max_side, Arena A)
{
    const int q = B.x * blockDim.x + threadIdx.x;
    if (q >= count) return;
    rr_instance *I = &inst[q];
    JobWS &ws = wsv[q];
    I->n_moves = 0; I->n_steps = 0; I->n_ops = 0; I->n_members = 0;
    I->status = RR_OK;
    const int m = I->m, n = I->n;
    const rr_rect R = I->rect;
    if (m < 1 || n < 1 || m > max_side || n > max_side || m > RR_MAX_SIDE || n > RR_MAX_SIDE || R.r0 < 0 || R.r0 >= R.r1 || R.r1 > m ||
        R.c0 < 0 || R.c0 >= R.c1 || R.c1 > n || !I->grid || (I->layout != RR_U8 && I->layout != RR_BITS32) ||
        I->cap_moves < 0 || (I->cap_moves > 0 && !I->moves)) {
        I->status = RR_ERR_ARG;
        return;
    }
    const int W = (m + 31) >> 5, h = R.r1 - R.r0, tw = R.c1 - R.c0;
    bool ok = true;
    ws.colbits = (uint32_t *)arena_alloc(A, sizeof(uint32_t) * (unsigned long long)n * W, &ok);
    ws.atomRows = (int16_t *)arena_alloc(A, sizeof(int16_t) * (unsigned long long)n * m, &ok);
    ws.holeRows = (int16_t *)arena_alloc(A, sizeof(int16_t) * (unsigned long long)tw * h, &ok);
    ws.col = (ColInfo *)arena_alloc(A, sizeof(ColInfo) * (unsigned long long)n, &ok);
    ws.recv = (RecvInfo *)arena_alloc(A, sizeof(RecvInfo) * (unsigned long long)n, &ok);
    ws.ev = (Event *)arena_alloc(A, sizeof(Event) * (unsigned long long)(n + 1), &ok);
    ws.unitOff = (int32_t *)arena_alloc(A, sizeof(int32_t) * (unsigned long long)(2 * n + 1), &ok);
    ws.nrecv = 0; ws.nev = 0;
    if (!ok) I->status = RR_ERR_WORKSPACE;
}

// ------------------------------------------------- S0: load and transpose
// Column-major bit columns: word w of column c holds rows 32w .. 32w+31.
// bits32 input, rows 16-byte aligned (a row length of a multiple of 128
// columns and an aligned grid): a warp takes 32 rows x 128 columns, lane l
// reads four words of row 32w + l in one 16-byte load, and each of the four
// 32x32 bit tiles is transposed with 32 ballots. Other rows: a warp takes
// one 32x32 tile, one word per lane.
// u8 input, rows 4-byte aligned: a warp takes 32 rows x 128 columns, lane l
// reads four consecutive bytes (columns 4l .. 4l+3) of each row in one
// 4-byte load, so that a warp reads 128 contiguous bytes per row, and builds
// its four columns' words. Other rows: lane l reads column 32g + l byte by
// byte (32 contiguous bytes per row and warp).
__device__ inline void s_transpose(const Blk B, rr_instance *inst, JobWS *wsv, int count)
{
    const int q = B.y;
    if (q >= count) return;
    const rr_instance *I = &inst[q];
    if (!live(I)) return;
    JobWS &ws = wsv[q];
    const int m = I->m, n = I->n, W = (m + 31) >> 5, G = (n + 31) >> 5, G4 = (n + 127) >> 7;
    const int lane = threadIdx.x & 31;
    const int w0 = B.x * (blockDim.x >> 5) + (threadIdx.x >> 5), nw = B.gx * (blockDim.x >> 5);
    if (I->layout == RR_BITS32) {
        const uint32_t *src = (const uint32_t *)I->grid;
        if ((G & 3) == 0 && ((uintptr_t)src & 15) == 0) {
            for (int item = w0; item < G4 * W; item += nw) {
                const int g4 = item / W, w = item % W;
                const int row = 32 * w + lane;
                uint4 v = make_uint4(0u, 0u, 0u, 0u);
                if (row < m) v = *reinterpret_cast<const uint4 *>(src + (size_t)row * G + 4 * g4);
                const uint32_t x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    uint32_t mine = 0;
#pragma unroll
                    for (int bt = 0; bt < 32; ++bt) {
                        const uint32_t bal = __ballot_sync(FULL, (x[c] >> bt) & 1u);
                        if (bt == lane) mine = bal;
                    }
                    const int col = 32 * (4 * g4 + c) + lane;
                    if (col < n) ws.colbits[(size_t)col * W + w] = mine;
                }
            }
        } else {
            for (int item = w0; item < G * W; item += nw) {
                const int g = item / W, w = item % W;
                const int row = 32 * w + lane;
                const uint32_t x = row < m ? src[(size_t)row * G + g] : 0u;
                uint32_t mine = 0;
#pragma unroll
                for (int bt = 0; bt < 32; ++bt) {
                    const uint32_t bal = __ballot_sync(FULL, (x >> bt) & 1u);
                    if (bt == lane) mine = bal;
                }
                const int col = 32 * g + lane;
                if (col < n) ws.colbits[(size_t)col * W + w] = mine;
            }
        }
    } else {
        const uint8_t *src = (const uint8_t *)I->grid;
        if ((n & 3) == 0 && ((uintptr_t)src & 3) == 0) {
            for (int item = w0; item < G4 * W; item += nw) {
                const int g4 = item / W, w = item % W;
                const int c0 = 128 * g4 + 4 * lane;
                if (c0 >= n) continue;
                const int rmax = min(32, m - 32 * w);
                const uint8_t *rp = src + (size_t)(32 * w) * n + c0;
                uint32_t a0 = 0u, a1 = 0u, a2 = 0u, a3 = 0u;
                for (int r = 0; r < rmax; ++r) {
                    const uint32_t v = *reinterpret_cast<const uint32_t *>(rp + (size_t)r * n);
                    a0 |= (uint32_t)((v & 0xffu) != 0u) << r;
                    a1 |= (uint32_t)((v & 0xff00u) != 0u) << r;
                    a2 |= (uint32_t)((v & 0xff0000u) != 0u) << r;
                    a3 |= (uint32_t)((v & 0xff000000u) != 0u) << r;
                }
                uint32_t *out = ws.colbits + (size_t)c0 * W + w;
                out[0] = a0;
                out[W] = a1;
                out[2 * W] = a2;
                out[3 * W] = a3;
            }
        } else {
            for (int item = w0; item < G * W; item += nw) {
                const int g = item / W, w = item % W;
                const int col = 32 * g + lane;
                if (col >= n) continue;
                const int rmax = min(32, m - 32 * w);
                uint32_t mine = 0;
                for (int r = 0; r < rmax; ++r) mine |= (uint32_t)(src[(size_t)(32 * w + r) * n + col] != 0) << r;
                ws.colbits[(size_t)col * W + w] = mine;
            }
        }
    }
}

// -------------------------------------- S1-S3: counts, surplus, column solves
// One warp per column. Target columns of non-negative surplus get the exact
// 1D solve: the h sources are the band atoms plus the a nearest atoms above
// and the x-a nearest below (a contiguous window of the sorted sources),
// a chosen by minimum total distance with the largest a on ties. Columns
// outside the target columns are pushed into their reservoir rows when they
// have the atoms for it, unless `strict` (then only their reservoir-row atoms
// are donatable and nothing in them moves).
__device__ inline void s_colstats(const Blk B, rr_instance *inst, JobWS *wsv, int count, int strict)
{
    const int q = B.y;
    if (q >= count) return;
    const rr_instance *I = &inst[q];
    if (!live(I)) return;
    JobWS &ws = wsv[q];
    const int m = I->m, n = I->n, W = (m + 31) >> 5;
    const int r0 = I->rect.r0, r1 = I->rect.r1, c0 = I->rect.c0, c1 = I->rect.c1;
    const int h = r1 - r0, R = m - h;
    const int lane = threadIdx.x & 31;
    const int nw = B.gx * (blockDim.x >> 5);
    for (int c = B.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < n; c += nw) {
        const uint32_t x = lane < W ? ws.colbits[(size_t)c * W + lane] : 0u;
        const uint32_t mT = row_mask(lane, 0, r0), mBd = row_mask(lane, r0, r1), mO = row_mask(lane, r1, m);
        const int cAll = __popc(x);
        const int incl = warp_incl_scan(cAll);
        const int K = __shfl_sync(FULL, incl, 31);
        const int ntop = warp_sum(__popc(x & mT));
        const int nband = warp_sum(__popc(x & mBd));
        const int nbot = warp_sum(__popc(x & mO));
        int16_t *rows = ws.atomRows + (size_t)c * m;
        {
            int p = incl - cAll;
            uint32_t y = x;
            while (y) { const int b = __ffs(y) - 1; rows[p++] = (int16_t)(32 * lane + b); y &= y - 1; }
        }
        const bool target = c >= c0 && c < c1;
        int16_t *hr = target ? ws.holeRows + (size_t)(c - c0) * h : nullptr;
        if (target) {
            uint32_t hx = ~x & mBd;
            const int ch = __popc(hx);
            int p = warp_incl_scan(ch) - ch;
            while (hx) { const int b = __ffs(hx) - 1; hr[p++] = (int16_t)(32 * lane + b); hx &= hx - 1; }
        }
        __syncwarp();

        ColInfo ci;
        ci.K = K; ci.ntop = ntop; ci.nband = nband; ci.nbot = nbot;
        ci.a = 0; ci.kd_end = 0; ci.ku_start = 0; ci.nmoves = 0; ci.topRun = 0; ci.botRun = 0;
        ci.tbase = 0; ci.bbase = 0;
        if (target) {
            ci.sigma = K - h;
            if (ci.sigma >= 0) {
                ci.kind = KIND_TARGET_SOLVED;
                const int need = h - nband, nh = h - nband;
                const int lo = max(0, need - nbot), hi = min(need, ntop);
                // d cost/da = (r0+a-1 - top(a-1)) + (2 P(r0+a-1) - M) + (r0+h-need+a-1 - bot(need-a))
                const int a = split_search(lo, hi, [&](int aa) {
                    const int topRow = rows[ntop - aa];                  // (aa-1)-th nearest above
                    const int botRow = rows[ntop + nband + (need - aa)]; // (need-aa)-th nearest below
                    return (r0 + aa - 1 - topRow) + (2 * band_P(hr, nh, nband, r0, r0 + aa - 1) - nband) +
                           (r0 + h - need + aa - 1 - botRow);
                });
                ci.a = a;
                ci.kd_end = a + band_P(hr, nh, nband, r0, r0 + a - 1);
                ci.ku_start = a + band_P(hr, nh, nband, r0, r0 + a);
                ci.nmoves = ci.kd_end + (h - ci.ku_start);
                ci.ptop = ntop - a;
                ci.pbot = nbot - (need - a);
                ci.tbase = ntop - a - 1;
                ci.bbase = ntop - a + h;
            } else {
                ci.kind = KIND_RECEIVER;
                ci.ptop = 0; ci.pbot = 0;
            }
        } else if (!strict && K >= R) {
            // Virtual targets = this column's reservoir cells: the first r0
            // atoms go to rows 0..r0-1, the last m-r1 to rows r1..m-1.
            ci.kind = KIND_OUTER_FULL;
            ci.sigma = R; ci.ptop = r0; ci.pbot = m - r1;
            const uint32_t valid = row_mask(lane, 0, m);
            const uint32_t brk = ~x | ~valid;                     // first non-atom from row 0
            const int fz = brk ? 32 * lane + __ffs(brk) - 1 : 0x7fffffff;
            int firstZero = fz;
#pragma unroll
            for (int o = 16; o; o >>= 1) firstZero = min(firstZero, __shfl_xor_sync(FULL, firstZero, o));
            if (firstZero > m) firstZero = m;
            const uint32_t z2 = ~x & valid;                       // last empty row
            int lz = z2 ? 32 * lane + 31 - __clz(z2) : -1;
#pragma unroll
            for (int o = 16; o; o >>= 1) lz = max(lz, __shfl_xor_sync(FULL, lz, o));
            ci.topRun = min(firstZero, r0);
            ci.botRun = min(m - 1 - lz, m - r1);
            ci.nmoves = (r0 - ci.topRun) + (m - r1 - ci.botRun);
        } else {
            ci.kind = KIND_OUTER_PART;
            ci.sigma = ntop + nbot; ci.ptop = ntop; ci.pbot = nbot;
            ci.tbase = ntop - 1; ci.bbase = ntop + nband;
        }
        if (lane == 0) ws.col[c] = ci;
    }
}

// ------------------------------------------------- S4: pairing (one warp)

struct PairSmem {
    int32_t *sig;
    int16_t *prv, *nxt, *tT, *bT, *mandT, *mandB, *evHead, *evTail, *evCnt;
    unsigned long long *score;
};

__device__ __forceinline__ unsigned long long pair_score(const PairSmem &S, int c)
{
    const int s1 = S.sig[c];
    if (s1 == 0) return 0ull;
    const int v = S.nxt[c];
    if (v < 0) return 0ull;
    const int s2 = S.sig[v];
    if ((s1 > 0) == (s2 > 0)) return 0ull;
    const int i = s1 > 0 ? c : v, j = s1 > 0 ? v : c;
    const int need = -S.sig[j];
    const int x = min(S.sig[i], need);
    const int d = iabs(i - j);
    const unsigned long long left = i < j ? 1ull : 0ull;
    // larger is better: tokens exchanged, then smaller gap, then smaller
    // deficit, then smaller receiver index, then smaller donor index.
    return ((unsigned long long)x << 42) | ((unsigned long long)(1023 - d) << 32) |
           ((unsigned long long)(2047 - need) << 21) | ((unsigned long long)(1023 - j) << 11) |
           (left << 10) | (unsigned long long)c;
}

__device__ inline void s_pair(const Blk B, rr_instance *inst, JobWS *wsv, int count)
{
    extern __shared__ unsigned long long smem_u64[];
    const int q = B.x;
    if (q >= count) return;
    rr_instance *I = &inst[q];
    if (!live(I)) return;
    JobWS &ws = wsv[q];
    const int m = I->m, n = I->n;
    const int r0 = I->rect.r0, r1 = I->rect.r1, c0 = I->rect.c0;
    const int h = r1 - r0;
    const int lane = threadIdx.x & 31;

    PairSmem S;
    S.score = smem_u64;
    S.sig = (int32_t *)(smem_u64 + n);
    S.prv = (int16_t *)(S.sig + n);
    S.nxt = S.prv + n; S.tT = S.nxt + n; S.bT = S.tT + n; S.mandT = S.bT + n; S.mandB = S.mandT + n;
    S.evHead = S.mandB + n; S.evTail = S.evHead + n; S.evCnt = S.evTail + n;

    int tot = 0, nneg = 0;
    for (int c = lane; c < n; c += 32) {
        const ColInfo ci = ws.col[c];
        S.sig[c] = ci.sigma;
        S.tT[c] = 0; S.bT[c] = 0;
        S.mandT[c] = (int16_t)ci.ntop; S.mandB[c] = (int16_t)ci.nbot;
        S.evHead[c] = -1; S.evTail[c] = -1; S.evCnt[c] = 0;
        tot += ci.sigma;
        nneg += ci.sigma < 0;
    }
    tot = warp_sum(tot);
    nneg = warp_sum(nneg);
    if (tot < 0) {                    // some column can never be saturated (Sec. III.C)
        if (lane == 0) { I->status = RR_INFEASIBLE; I->n_moves = 0; }
        return;
    }
    __syncwarp();
    // list of non-zero-surplus columns: next (right-to-left sweep) and prev
    {
        int carry = -1;
        for (int base = ((n - 1) >> 5) << 5; base >= 0; base -= 32) {
            const int c = base + lane;
            const unsigned nz = __ballot_sync(FULL, c < n && S.sig[c] != 0);
            const unsigned above = lane < 31 ? nz & ~((2u << lane) - 1u) : 0u;
            if (c < n) S.nxt[c] = (int16_t)(above ? base + __ffs(above) - 1 : carry);
            if (nz) carry = base + __ffs(nz) - 1;
        }
        carry = -1;
        for (int base = 0; base < n; base += 32) {
            const int c = base + lane;
            const unsigned nz = __ballot_sync(FULL, c < n && S.sig[c] != 0);
            const unsigned below = nz & ((1u << lane) - 1u);
            if (c < n) S.prv[c] = (int16_t)(below ? base + 31 - __clz(below) : carry);
            if (nz) carry = base + 31 - __clz(nz);
        }
    }
    __syncwarp();
    for (int c = lane; c < n; c += 32) S.score[c] = pair_score(S, c);
    __syncwarp();

    int nrecv = 0, nev = 0;
    const int16_t *allRows = ws.atomRows;
    for (int iter = 0; nneg > 0; ++iter) {
        if (iter > n || (g_guard_cap > 0 && iter >= g_guard_cap)) { if (lane == 0) I->status = RR_ERR_TIMEOUT; return; }
        unsigned long long best = 0ull;
        for (int c = lane; c < n; c += 32) { const unsigned long long s = S.score[c]; best = s > best ? s : best; }
        best = warp_max_u64(best);
        if (best == 0ull) { if (lane == 0) I->status = RR_ERR_INTERNAL; return; }
        const int cpos = (int)(best & 1023ull);
        const int other = S.nxt[cpos];
        const int i = S.sig[cpos] > 0 ? cpos : other;
        const int j = S.sig[cpos] > 0 ? other : cpos;
        const int si = S.sig[i], need = -S.sig[j];
        const int x = min(si, need);
        const int kase = si > need ? 1 : (si == need ? 2 : 3);
        const ColInfo D = ws.col[i];
        const int16_t *drows = allRows + (size_t)i * m;
        const int t0 = S.tT[i], b0 = S.bT[i];
        const int availT = D.ptop - t0, availB = D.pbot - b0;
        const int e = nev++;
        Event ev;
        ev.kase = kase; ev.i = i; ev.j = j; ev.x = x; ev.t0 = t0; ev.b0 = b0; ev.next = -1;
        if (kase == 3) {
            ev.a = availT;
            if (lane == 0) {
                S.mandT[j] += (int16_t)availT; S.mandB[j] += (int16_t)availB;
                S.tT[i] = (int16_t)D.ptop; S.bT[i] = (int16_t)D.pbot;
                S.sig[j] += si; S.sig[i] = 0;
            }
        } else {
            const int mT = S.mandT[j], mB = S.mandB[j];
            const ColInfo Rj = ws.col[j];
            const int M = Rj.nband, nh = h - M;
            const int16_t *hr = ws.holeRows + (size_t)(j - c0) * h;
            int a;
            if (kase == 2) {
                a = availT;
                if (availT + availB != x) { if (lane == 0) I->status = RR_ERR_INTERNAL; return; }
            } else {
                const int lo = max(0, x - availB), hi = min(x, availT);
                a = split_search(lo, hi, [&](int aa) {
                    const int tr = pool_top_row(D, drows, r0, t0 + aa - 1);
                    const int br = pool_bot_row(D, drows, r1, b0 + x - aa);
                    return (r0 + mT + aa - 1 - tr) + (2 * band_P(hr, nh, M, r0, r0 + mT + aa - 1) - M) +
                           (r0 + h - mB - x + aa - 1 - br);
                });
            }
            ev.a = a;
            const int nT = mT + a;
            RecvInfo ri;
            ri.j = j;
            ri.nT = nT;
            ri.kd_end = nT + band_P(hr, nh, M, r0, r0 + nT - 1);
            ri.ku_start = nT + band_P(hr, nh, M, r0, r0 + nT);
            ri.nmoves = ri.kd_end + (h - ri.ku_start);
            ri.pad = 0;
            if (lane == 0) {
                S.tT[i] = (int16_t)(t0 + a); S.bT[i] = (int16_t)(b0 + x - a);
                S.sig[i] -= x; S.sig[j] = 0;
                // link this event, then close the receiver's list
                if (S.evTail[j] >= 0) ws.ev[S.evTail[j]].next = e; else S.evHead[j] = (int16_t)e;
                S.evTail[j] = (int16_t)e; S.evCnt[j] += 1;
                ri.ev_first = S.evHead[j];
                ri.ncontrib = S.evCnt[j];
                ws.recv[nrecv] = ri;
            }
            ++nrecv;
            --nneg;
        }
        if (lane == 0) {
            if (kase == 3) {
                if (S.evTail[j] >= 0) ws.ev[S.evTail[j]].next = e; else S.evHead[j] = (int16_t)e;
                S.evTail[j] = (int16_t)e; S.evCnt[j] += 1;
            }
            ws.ev[e] = ev;
            // unlink columns that reached zero and refresh the scores around them
            int touched[6]; int nt = 0;
            const int cols2[2] = {i, j};
            for (int u = 0; u < 2; ++u) {
                const int c = cols2[u];
                if (S.sig[c] == 0) {
                    const int p = S.prv[c], nx = S.nxt[c];
                    if (p >= 0) S.nxt[p] = (int16_t)nx;
                    if (nx >= 0) S.prv[nx] = (int16_t)p;
                    S.score[c] = 0ull;
                    if (p >= 0) touched[nt++] = p;
                } else {
                    touched[nt++] = c;
                    if (S.prv[c] >= 0) touched[nt++] = S.prv[c];
                }
            }
            for (int u = 0; u < nt; ++u) S.score[touched[u]] = pair_score(S, touched[u]);
        }
        __syncwarp();
    }
    // move offsets of all solve units: column units in column order, then
    // receiver units in saturation order
    int carry = 0;
    const int U = n + nrecv;
    for (int base = 0; base < U; base += 32) {
        const int u = base + lane;
        int v = 0;
        if (u < n) v = ws.col[u].nmoves;
        else if (u < U) v = ws.recv[u - n].nmoves;
        const int incl = warp_incl_scan(v);
        if (u < U) ws.unitOff[u] = carry + incl - v;
        carry += __shfl_sync(FULL, incl, 31);
    }
    if (lane == 0) {
        ws.unitOff[U] = carry;
        ws.nrecv = nrecv;
        ws.nev = nev;
        I->n_moves = carry;
        if ((int64_t)carry > I->cap_moves) I->status = RR_ERR_CAPACITY;
    }
}

// ------------------------------------------------------ S6: column units

__device__ inline void s_emit_cols(const Blk B, rr_instance *inst, JobWS *wsv, int count)
{
    const int q = B.y;
    if (q >= count) return;
    rr_instance *I = &inst[q];
    if (!live(I)) return;
    JobWS &ws = wsv[q];
    const int m = I->m, n = I->n;
    const int r0 = I->rect.r0, r1 = I->rect.r1, h = r1 - r0;
    const int lane = threadIdx.x & 31;
    const int nw = B.gx * (blockDim.x >> 5);
    rr_move *out = I->moves;
    long long steps = 0;
    for (int c = B.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < n; c += nw) {
        const ColInfo ci = ws.col[c];
        if (ci.nmoves == 0) continue;
        const int16_t *rows = ws.atomRows + (size_t)c * m;
        rr_move *o = out + ws.unitOff[c];
        if (ci.kind == KIND_TARGET_SOLVED) {
            const int w = ci.ntop - ci.a;
            for (int k = lane; k < h; k += 32) {
                const int s = rows[w + k];
                int pos;
                if (k < ci.kd_end) pos = ci.kd_end - 1 - k;                  // toward larger rows, deepest first
                else if (k >= ci.ku_start) pos = ci.kd_end + (k - ci.ku_start);  // toward smaller rows
                else continue;                                                // isolated
                o[pos] = rr_move{s, c, r0 + k, c};
                steps += iabs(r0 + k - s);
            }
        } else {   // KIND_OUTER_FULL
            const int nbg = m - r1, ndown = nbg - ci.botRun;
            for (int k = lane; k < ndown; k += 32) {
                o[ndown - 1 - k] = rr_move{rows[ci.K - nbg + k], c, r1 + k, c};
                steps += r1 + k - rows[ci.K - nbg + k];
            }
            for (int k = ci.topRun + lane; k < r0; k += 32) {
                o[ndown + (k - ci.topRun)] = rr_move{rows[k], c, k, c};
                steps += rows[k] - k;
            }
        }
    }
    add_steps(I, steps);
}

// ---------------------------------------------------- S5/S6: receiver units

struct Contrib {
    int32_t col, kind, tbase, bbase;
    int32_t tStart, tCnt, bStart, bCnt;
    int32_t d, right, first;     // distance, right-side donor, first source index
};

// Top-region order at equal rows: farther column first, right before left.
__device__ __forceinline__ bool top_before(const Contrib &a, const Contrib &b)
{
    return a.d > b.d || (a.d == b.d && a.right && !b.right);
}
// Bottom-region order at equal rows: nearer column first, left before right.
__device__ __forceinline__ bool bot_before(const Contrib &a, const Contrib &b)
{
    return a.d < b.d || (a.d == b.d && !a.right && b.right);
}

constexpr int MAX_CONTRIB = 1024;

__device__ inline void s_emit_recv(const Blk B, rr_instance *inst, JobWS *wsv, int count)
{
    __shared__ Contrib C[MAX_CONTRIB + 1];
    __shared__ int s_nc;
    const int q = B.y;
    if (q >= count) return;
    rr_instance *I = &inst[q];
    if (!live(I)) return;
    JobWS &ws = wsv[q];
    const int m = I->m, n = I->n;
    const int r0 = I->rect.r0, r1 = I->rect.r1, h = r1 - r0;
    long long steps = 0;
    for (int r = B.x; r < ws.nrecv; r += B.gx) {
        const RecvInfo ri = ws.recv[r];
        const int j = ri.j;
        const ColInfo Rj = ws.col[j];
        const int16_t *own = ws.atomRows + (size_t)j * m;
        __syncthreads();
        if (threadIdx.x == 0) {
            int nc = 0, first = Rj.K, e = ri.ev_first;
            for (int u = 0; u < ri.ncontrib && e >= 0 && nc < MAX_CONTRIB; ++u) {
                const Event ev = ws.ev[e];
                const ColInfo D = ws.col[ev.i];
                Contrib c;
                c.col = ev.i; c.kind = D.kind; c.tbase = D.tbase; c.bbase = D.bbase;
                c.tStart = ev.t0; c.bStart = ev.b0;
                if (ev.kase == 3) { c.tCnt = D.ptop - ev.t0; c.bCnt = D.pbot - ev.b0; }
                else { c.tCnt = ev.a; c.bCnt = ev.x - ev.a; }
                c.d = iabs(ev.i - j); c.right = ev.i > j; c.first = first;
                first += c.tCnt + c.bCnt;
                C[nc++] = c;
                e = ev.next;
            }
            if (first != h || nc != ri.ncontrib) set_status(I, RR_ERR_INTERNAL);
            s_nc = nc;
        }
        __syncthreads();
        if (!live(I)) break;
        const int nc = s_nc;
        rr_move *o = I->moves + ws.unitOff[n + r];
        const int ownTop = Rj.ntop, ownBand = Rj.nband;
        for (int t = threadIdx.x; t < h; t += blockDim.x) {
            int row, col, ci = -1;
            if (t < Rj.K) { row = own[t]; col = j; }
            else {
                int lo = 0, hi = nc - 1;                 // contributor holding source t
                while (lo < hi) { const int mid = (lo + hi + 1) >> 1; if (C[mid].first <= t) lo = mid; else hi = mid - 1; }
                ci = lo;
                const Contrib &c = C[ci];
                const int u = t - c.first;
                const int16_t *drows = ws.atomRows + (size_t)c.col * m;
                if (u < c.tCnt) {
                    const int l = c.tStart + u;
                    row = c.kind == KIND_OUTER_FULL ? r0 - 1 - l : drows[c.tbase - l];
                } else {
                    const int l = c.bStart + (u - c.tCnt);
                    row = c.kind == KIND_OUTER_FULL ? r1 + l : drows[c.bbase + l];
                }
                col = c.col;
            }
            int k;
            if (row >= r0 && row < r1) {
                k = ri.nT + (t - ownTop);                 // own band atom (only own atoms sit in the band)
            } else {
                const bool top = row < r0;
                int below = 0, tie = 0;
                Contrib self;
                if (ci < 0) {
                    // own atom: own rows of its region before it are the ones before it in index
                    below = top ? t : t - ownTop - ownBand;
                    self.d = 0; self.right = 0;
                } else {
                    self = C[ci];
                    const int lo0 = top ? 0 : ownTop + ownBand, hi0 = top ? ownTop : Rj.K;
                    int lo = lo0, hi = hi0;
                    while (lo < hi) { const int mid = (lo + hi) >> 1; if (own[mid] < row) lo = mid + 1; else hi = mid; }
                    below = lo - lo0;
                    // the own atom (distance 0) comes first below the band, last above it
                    if (!top && lo < hi0 && own[lo] == row) ++tie;
                    // this contributor's other sources on the same side: nearest-first
                    // order is descending rows above the band, ascending below it
                    const int u = t - self.first;
                    below += top ? self.tCnt - 1 - u : u - self.tCnt;
                }
                for (int v = 0; v < nc; ++v) {
                    if (v == ci) continue;
                    const Contrib &c = C[v];
                    const int16_t *drows = ws.atomRows + (size_t)c.col * m;
                    if (top) {
                        int lo = c.tStart, hi = c.tStart + c.tCnt;   // first l with row(l) < row
                        while (lo < hi) {
                            const int mid = (lo + hi) >> 1;
                            const int rw = c.kind == KIND_OUTER_FULL ? r0 - 1 - mid : drows[c.tbase - mid];
                            if (rw < row) hi = mid; else lo = mid + 1;
                        }
                        below += c.tStart + c.tCnt - lo;
                        if (lo > c.tStart) {
                            const int l = lo - 1;
                            const int rw = c.kind == KIND_OUTER_FULL ? r0 - 1 - l : drows[c.tbase - l];
                            if (rw == row && top_before(c, self)) ++tie;
                        }
                    } else {
                        int lo = c.bStart, hi = c.bStart + c.bCnt;   // first l with row(l) >= row
                        while (lo < hi) {
                            const int mid = (lo + hi) >> 1;
                            const int rw = c.kind == KIND_OUTER_FULL ? r1 + mid : drows[c.bbase + mid];
                            if (rw < row) lo = mid + 1; else hi = mid;
                        }
                        below += lo - c.bStart;
                        if (lo < c.bStart + c.bCnt) {
                            const int rw = c.kind == KIND_OUTER_FULL ? r1 + lo : drows[c.bbase + lo];
                            if (rw == row && bot_before(c, self)) ++tie;
                        }
                    }
                }
                k = top ? below + tie : ri.nT + ownBand + below + tie;
            }
            if (k < 0 || k >= h) { set_status(I, RR_ERR_INTERNAL); continue; }
            int pos;
            if (k < ri.kd_end) pos = ri.kd_end - 1 - k;
            else if (k >= ri.ku_start) pos = ri.kd_end + (k - ri.ku_start);
            else continue;                                 // isolated own band atom
            if (pos >= ri.nmoves) { set_status(I, RR_ERR_INTERNAL); continue; }
            o[pos] = rr_move{row, col, r0 + k, j};
            steps += iabs(r0 + k - row) + iabs(j - col);
        }
    }
    add_steps(I, steps);
}

} // namespace rrk
