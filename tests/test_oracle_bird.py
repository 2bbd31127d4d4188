"""Pins of the bird oracle (Alg. 2, Sec. III.E) against facts fixed outside it.

- Validity (Sec. II.B-C): the move list replays without obstruction and fills
  the target; the feasibility condition is red-rec's (total surplus >= 0).
- Each receiver unit solves its column optimally over the tokens the
  generalised 1D instance may use (the column's own atoms and every atom in a
  reservoir row of another column, Sec. III.E): its total Manhattan length
  equals the minimum-cost assignment computed by scipy's solver on true
  Manhattan distances, which knows nothing of diagonals or windows.
- The column phase is red-rec's (Alg. 2 first steps = Alg. 1 first loop):
  without receivers the two planners give the same moves; with receivers the
  column-phase prefixes agree.
- Every token moves at most once, except atoms of columns outside the target
  columns (pushed into their reservoir rows first).
Hand-worked fixtures (tests/golden/bird_*.json) pin the tie rules."""
import numpy as np
import pytest

import oracle
from gridgen import square_instance, paper_instance, grid_u8, threshold
from tests.checks import replay_moves, assert_target_full, path_len


def _instances():
    out = []
    for seed in range(60):
        side = 6 + seed % 19
        out.append(square_instance(seed, 3, side, 0.5 + 0.05 * (seed % 4)))
    for seed in range(20):
        out.append(paper_instance(seed, 5, 6 + seed % 12))
    return out


def _rect_instances():
    """Rectangular grids with off-centre target rectangles (the readings do
    not need a centred target)."""
    rng = np.random.default_rng(11)
    out = []
    for seed in range(40):
        m, n = int(rng.integers(4, 20)), int(rng.integers(3, 20))
        r0 = int(rng.integers(0, m)); r1 = int(rng.integers(r0 + 1, m + 1))
        c0 = int(rng.integers(0, n)); c1 = int(rng.integers(c0 + 1, n + 1))
        p = float(rng.uniform(0.45, 0.8))
        out.append((grid_u8(seed, 7, m, n, threshold(p)), (r0, c0, r1, c1)))
    return out


def _all():
    return [(i.grid, i.rect) for i in _instances()] + _rect_instances()


def _units(moves, units):
    """Split a bird move list into (column-phase prefix, [unit moves...])."""
    moves = np.asarray(moves).reshape(-1, 4)
    k, spans = 0, []
    first = int(units[0][0]) if len(units) else None
    while k < len(moves) and (first is None or moves[k, 3] != first):
        k += 1
    prefix = moves[:k]
    for (j, _, _) in units:
        s = k
        while k < len(moves) and moves[k, 3] == j:
            k += 1
        spans.append((int(j), moves[s:k]))
    assert k == len(moves), "moves after the last receiver unit"
    return prefix, spans


@pytest.mark.parametrize("idx", range(100))
def test_bird_valid_and_feasibility_as_redrec(idx):
    grid, rect = _all()[idx]
    b = oracle.bird(grid, rect)
    r = oracle.plan(grid, rect)
    assert b.status == r.status
    if b.status == oracle.INFEASIBLE:
        assert len(b.moves) == 0
        return
    final = replay_moves(grid, rect, b.moves)
    assert_target_full(final, rect, grid)


@pytest.mark.parametrize("idx", range(100))
def test_bird_units_optimal(idx):
    from scipy.optimize import linear_sum_assignment
    grid, rect = _all()[idx]
    r0, c0, r1, c1 = rect
    m, n = grid.shape
    b = oracle.bird(grid, rect, with_trace=True)
    if b.status != 0:
        return
    prefix, spans = _units(b.moves, b.events)
    state = replay_moves(grid, rect, prefix) if len(prefix) else grid.copy()
    for (j, ntop, nbot), (jj, u) in zip(b.events, spans):
        assert j == jj and len(u) >= 1
        # candidates: the column's own atoms, reservoir-row atoms elsewhere
        cand = [(r, c) for r in range(m) for c in range(n) if state[r, c] and
                (c == j or r < r0 or r >= r1)]
        cost = np.array([[abs(r - t) + abs(c - j) for t in range(r0, r1)] for (r, c) in cand])
        ri, ci = linear_sum_assignment(cost)
        best = int(cost[ri, ci].sum())
        assert path_len(u) == best, (j, path_len(u), best)
        srcs = {(int(a), int(bb)) for a, bb, _, _ in u}
        assert srcs <= set(cand)
        # the unit's tokens from above / below the band match the trace
        assert sum(1 for (a, bb) in srcs if a < r0) == ntop
        assert sum(1 for (a, bb) in srcs if a >= r1) == nbot
        state = replay_moves(state, rect, u)
        assert state[r0:r1, j].all()


@pytest.mark.parametrize("idx", range(100))
def test_bird_column_phase_is_redrecs(idx):
    grid, rect = _all()[idx]
    b = oracle.bird(grid, rect, with_trace=True)
    r = oracle.plan(grid, rect, with_trace=True)
    if b.status != 0:
        return
    if len(b.events) == 0:
        assert len(r.events) == 0
        assert b.moves.tolist() == r.moves.tolist()
        return
    prefix, _ = _units(b.moves, b.events)
    assert r.moves[: len(prefix)].tolist() == prefix.tolist()
    # red-rec's next move belongs to a receiver unit (not its column phase)
    rec = {int(e[2]) for e in r.events}
    if len(r.moves) > len(prefix):
        assert int(r.moves[len(prefix), 3]) in rec


@pytest.mark.parametrize("idx", range(100))
def test_bird_each_token_moves_once(idx):
    grid, rect = _all()[idx]
    r0, c0, r1, c1 = rect
    b = oracle.bird(grid, rect)
    if b.status != 0:
        return
    arrived = {}
    for k, (sr, sc, dr, dc) in enumerate(b.moves.tolist()):
        if (sr, sc) in arrived:
            assert not (c0 <= sc < c1), f"move {k}: an atom of target column {sc} moves twice"
        arrived[(dr, dc)] = k


def test_bird_no_receiver_equals_redrec():
    """A fully loaded grid has no receiver: both planners reduce to the
    column phase."""
    for side in (5, 9, 16):
        grid = np.ones((side, side), dtype=np.uint8)
        grid[0, :] = 0
        rect = (1, 1, side - 1, side - 1)
        b = oracle.bird(grid, rect, with_trace=True)
        r = oracle.plan(grid, rect)
        assert len(b.events) == 0 and b.status == r.status == 0
        assert b.moves.tolist() == r.moves.tolist()


def test_bird_infeasible():
    grid = np.zeros((6, 6), dtype=np.uint8)
    grid[2, 1] = 1
    b = oracle.bird(grid, (1, 1, 5, 5))
    assert b.status == oracle.INFEASIBLE and len(b.moves) == 0


def test_bird_prefers_nearby_tokens_over_one_donor():
    """The situation Sec. III.E uses to motivate bird, at random: summed over
    many grids, bird's receiver units are never longer than an optimal
    assignment (pinned above) and red-rec's one-donor units are at least as
    long as bird's when both start from the same state (a single receiver)."""
    rng = np.random.default_rng(5)
    checked = 0
    for t in range(200):
        m, n = 9, 3
        grid = np.zeros((m, n), dtype=np.uint8)
        rect = (3, 0, 6, 3)
        grid[3:6, 0] = 1; grid[3:6, 2] = 1
        grid[int(rng.integers(3, 6)), 1] = 1
        for c in (0, 2):
            for r in list(range(0, 3)) + list(range(6, 9)):
                grid[r, c] = rng.random() < 0.4
        b = oracle.bird(grid, rect)
        r = oracle.plan(grid, rect)
        if b.status or r.status:
            continue
        checked += 1
        assert path_len(b.moves) <= path_len(r.moves)
    assert checked > 50


def test_bird_prefix_is_a_prefix():
    """rro_bird_prefix (used for full-size sampled parity) stops after its
    first receiver units: its moves are the leading moves of the full plan."""
    for seed in range(12):
        inst = square_instance(seed, 21, 24 + seed, 0.55)
        full = oracle.bird(inst.grid, inst.rect, with_trace=True)
        if full.status != 0:
            continue
        for u in (0, 1, 2, len(full.events)):
            p = oracle.bird_prefix(inst.grid, inst.rect, u)
            assert p.moves.tolist() == full.moves[: len(p.moves)].tolist()
        assert len(oracle.bird_prefix(inst.grid, inst.rect, len(full.events)).moves) == len(full.moves)
