"""Independent checkers used by the tests: they restate the paper's validity
conditions directly (Sec. II.B-C: an unobstructed move needs every vertex of
its path other than the source free of tokens; a valid path system fills T;
Alg. 4: a batch holds at most one next edge per path, pairwise disjoint; Sec.
IV: every pair of tokens in a batch moves in the same direction and shares a
row or a column). They share no code with the oracle or the CUDA library.
"""
from __future__ import annotations

import numpy as np

DIRS = {0: (-1, 0), 1: (1, 0), 2: (0, -1), 3: (0, 1)}


def path_cells(mv):
    """Vertices of the shortest path of a move, row first then column."""
    sr, sc, dr, dc = (int(v) for v in mv)
    cells = []
    step = 1 if dc >= sc else -1
    for c in range(sc, dc + step, step):
        cells.append((sr, c))
    step = 1 if dr >= sr else -1
    for r in range(sr + step, dr + step, step):
        cells.append((r, dc))
    return cells


def path_len(moves) -> int:
    mv = np.asarray(moves, dtype=np.int64).reshape(-1, 4)
    return int((np.abs(mv[:, 0] - mv[:, 2]) + np.abs(mv[:, 1] - mv[:, 3])).sum())


def replay_moves(grid, rect, moves):
    """Execute the moves in list order; every move must be unobstructed.
    Returns the final occupancy grid."""
    g = np.array(grid, dtype=np.uint8, copy=True)
    for idx, mv in enumerate(np.asarray(moves).reshape(-1, 4)):
        cells = path_cells(mv)
        assert len(cells) >= 2, f"move {idx} is isolated"
        r, c = cells[0]
        assert g[r, c] == 1, f"move {idx}: no atom at source {cells[0]}"
        for (rr, cc) in cells[1:]:
            assert g[rr, cc] == 0, f"move {idx}: collision at {(rr, cc)}"
        g[r, c] = 0
        g[cells[-1]] = 1
    return g


def assert_target_full(final, rect, initial):
    r0, c0, r1, c1 = rect
    assert final[r0:r1, c0:c1].all(), "target not fully occupied"
    assert int(final.sum()) == int(np.asarray(initial).sum()), "atom count not conserved"


def replay_ops(grid, moves, ops, members):
    """Execute batches: each op moves every member one elementary step along
    its own path. Checks the per-batch rules and that every path is executed
    completely. Returns the final grid."""
    moves = np.asarray(moves).reshape(-1, 4)
    g = np.array(grid, dtype=np.uint8, copy=True)
    cells = [path_cells(mv) for mv in moves]
    prog = [0] * len(moves)
    for oi, (d, first, count) in enumerate(np.asarray(ops).reshape(-1, 3)):
        mem = [int(v) for v in members[first:first + count]]
        assert count >= 1, f"op {oi} empty"
        assert mem == sorted(set(mem)), f"op {oi}: members not strictly ascending"
        tails, heads = [], []
        for b in mem:
            cl = cells[b]
            t = prog[b]
            assert t < len(cl) - 1, f"op {oi}: path {b} already finished"
            (r, c), (r2, c2) = cl[t], cl[t + 1]
            assert (r2 - r, c2 - c) == DIRS[int(d)], f"op {oi}: path {b} does not step in dir {d}"
            tails.append((r, c))
            heads.append((r2, c2))
        # same line: every pair shares a row or a column
        for i in range(len(tails)):
            for j in range(i + 1, len(tails)):
                a, b = tails[i], tails[j]
                assert a[0] == b[0] or a[1] == b[1], f"op {oi}: tokens {a} {b} not on one line"
        # edges pairwise disjoint, destinations free before the batch
        verts = tails + heads
        assert len(set(verts)) == len(verts), f"op {oi}: edges intersect"
        for (r, c) in tails:
            assert g[r, c] == 1, f"op {oi}: no atom at {(r, c)}"
        for (r, c) in heads:
            assert g[r, c] == 0, f"op {oi}: collision at {(r, c)}"
        for (r, c) in tails:
            g[r, c] = 0
        for (r, c) in heads:
            g[r, c] = 1
        for b in mem:
            prog[b] += 1
    for b, cl in enumerate(cells):
        assert prog[b] == len(cl) - 1, f"path {b} not completed ({prog[b]} of {len(cl) - 1})"
    return g


def batch_bruteforce(moves):
    """Alg. 4 with Gamma taken literally: a path is ready iff no earlier
    unfinished path shares a vertex with it; ready paths are visited in id
    order and a next step joins iff it has the first member's direction and
    its token shares a row or a column with every member's token. Quadratic;
    tiny inputs only."""
    moves = np.asarray(moves).reshape(-1, 4)
    k = len(moves)
    cells = [path_cells(mv) for mv in moves]
    sets = [set(c) for c in cells]
    prog = [0] * k
    done = [False] * k
    ops, members = [], []
    while not all(done):
        Q = [b for b in range(k) if not done[b]
             and not any((not done[a]) and (sets[a] & sets[b]) for a in range(b))]
        assert Q, "deadlock"
        acc, d0 = [], None
        for b in Q:
            (r, c), (r2, c2) = cells[b][prog[b]], cells[b][prog[b] + 1]
            d = {v: kk for kk, v in DIRS.items()}[(r2 - r, c2 - c)]
            if not acc:
                acc.append((b, r, c)); d0 = d
            elif d == d0 and all(ar == r or ac == c for (_, ar, ac) in acc):
                acc.append((b, r, c))
        ops.append((d0, len(members), len(acc)))
        for (b, _, _) in acc:
            members.append(b)
            prog[b] += 1
            if prog[b] == len(cells[b]) - 1:
                done[b] = True
    return np.array(ops, dtype=np.int32).reshape(-1, 3), np.array(members, dtype=np.int32)


def grid_from_rows(rows):
    return np.array([[1 if ch == "#" else 0 for ch in row] for row in rows], dtype=np.uint8)
