"""The oracle against hand-worked instances (tests/golden/*.json).

Each fixture was solved by hand from the rules of Alg. 1 / Sec. III.A-C,
Alg. 2 / Sec. III.E (fixtures with "planner": "bird") and Alg. 4 / Sec. IV,
with the derivation written in the file."""
import glob
import json
import os

import pytest

import oracle
from tests.checks import grid_from_rows, replay_moves, assert_target_full, replay_ops

GOLDEN = sorted(glob.glob(os.path.join(os.path.dirname(__file__), "golden", "*.json")))


@pytest.mark.parametrize("path", GOLDEN, ids=[os.path.basename(p)[:-5] for p in GOLDEN])
def test_golden(path):
    fx = json.load(open(path))
    grid = grid_from_rows(fx["grid"])
    rect = tuple(fx["rect"])
    if fx.get("planner") == "bird":
        p = oracle.bird(grid, rect, with_trace=True)
        assert p.events.tolist() == fx["units"]
    else:
        p = oracle.plan(grid, rect, with_trace=True)
        assert p.events.tolist() == fx["events"]
    assert p.status == fx["status"]
    assert p.moves.tolist() == fx["moves"]
    ops, mem = oracle.batch(p.moves, *grid.shape)
    assert ops.tolist() == fx["ops"]
    assert mem.tolist() == fx["members"]
    if p.status == 0:
        final = replay_moves(grid, rect, p.moves)
        assert_target_full(final, rect, grid)
        assert (replay_ops(grid, p.moves, ops, mem) == final).all()


def test_golden_fixture_count():
    assert len(GOLDEN) >= 10
