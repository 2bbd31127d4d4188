"""Pins of the strict-reservoir reading of target sub-rectangles (columns
outside the target columns donate only the atoms already in their reservoir
rows; Sec. III.C: donors give reservoir atoms only), for red-rec and bird.

- With a full-width target there are no outer columns: both readings are the
  paper's algorithm and give identical plans.
- Every token moves at most once (Sec. III.C states this for red-rec; under
  this reading it holds without exception), and nothing in an outer column
  ever moves but its reservoir-row atoms.
- Feasibility is the total surplus computed here from its definition: target
  columns K - h, outer columns their reservoir-row atoms.
- The counting argument for a centred square target of 0.7 times the side at
  fill 0.6: the target columns miss t(t - p s) atoms on average against
  p (s - t)^2 reservoir atoms of the outer columns, so 256 x 256 grids with a
  180 x 180 target are infeasible.
"""
import numpy as np
import pytest

import oracle
from gridgen import square_instance, paper_instance, grid_u8, threshold
from tests.checks import replay_moves, assert_target_full


def _cases():
    rng = np.random.default_rng(23)
    out = []
    for seed in range(60):
        m, n = int(rng.integers(4, 24)), int(rng.integers(4, 24))
        r0 = int(rng.integers(0, m)); r1 = int(rng.integers(r0 + 1, m + 1))
        c0 = int(rng.integers(0, n)); c1 = int(rng.integers(c0 + 1, n + 1))
        out.append((grid_u8(seed, 13, m, n, threshold(float(rng.uniform(0.5, 0.9)))), (r0, c0, r1, c1)))
    return out


def _strict_surplus(grid, rect):
    r0, c0, r1, c1 = rect
    h = r1 - r0
    tot = 0
    for c in range(grid.shape[1]):
        col = grid[:, c]
        if c0 <= c < c1:
            tot += int(col.sum()) - h
        else:
            tot += int(col[:r0].sum() + col[r1:].sum())
    return tot


@pytest.mark.parametrize("planner", ["plan", "bird"])
def test_full_width_readings_agree(planner):
    f = getattr(oracle, planner)
    for seed in range(30):
        inst = paper_instance(seed, 3, 6 + seed % 20)
        a, b = f(inst.grid, inst.rect), f(inst.grid, inst.rect, strict=True)
        assert a.status == b.status and a.moves.tolist() == b.moves.tolist()


@pytest.mark.parametrize("planner", ["plan", "bird"])
@pytest.mark.parametrize("idx", range(60))
def test_strict_valid_once_and_feasibility(planner, idx):
    grid, rect = _cases()[idx]
    r0, c0, r1, c1 = rect
    p = getattr(oracle, planner)(grid, rect, strict=True)
    feasible = _strict_surplus(grid, rect) >= 0
    assert p.status == (oracle.OK if feasible else oracle.INFEASIBLE)
    if not feasible:
        assert len(p.moves) == 0
        return
    final = replay_moves(grid, rect, p.moves)
    assert_target_full(final, rect, grid)
    moved_to = set()
    for (sr, sc, dr, dc) in p.moves.tolist():
        assert (sr, sc) not in moved_to, "a token moved twice"
        moved_to.add((dr, dc))
        if not (c0 <= sc < c1):
            assert sr < r0 or sr >= r1, "an outer column's band-row atom moved"
        assert c0 <= dc < c1, "a move ends outside the target columns"


def test_strict_square_target_infeasible_at_fill_06():
    for seed in range(4):
        inst = square_instance(seed, 0, 256, 0.6, 180)
        assert _strict_surplus(inst.grid, inst.rect) < 0
        assert oracle.plan(inst.grid, inst.rect, strict=True).status == oracle.INFEASIBLE
        assert oracle.plan(inst.grid, inst.rect).status == oracle.OK
