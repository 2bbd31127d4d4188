"""The GPU path against the hand-worked fixtures (tests/golden/*.json): moves,
batches and members equal the values derived by hand from the paper's rules,
with no oracle in between (red-rec fixtures through rr_plan, bird fixtures
through rr_bird_plan, both layouts; the batches through rr_batch)."""
import glob
import json
import os

import numpy as np
import pytest

import gridgen
from tests.checks import grid_from_rows

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

GOLDEN = sorted(glob.glob(os.path.join(os.path.dirname(__file__), "golden", "*.json")))


@pytest.fixture(scope="module")
def planner():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_06182_gb300.planner import Planner
    p = Planner(arena_bytes=256 << 20)
    yield p
    p.close()


@pytest.mark.parametrize("path", GOLDEN, ids=[os.path.basename(p)[:-5] for p in GOLDEN])
def test_gpu_equals_hand_worked_fixture(planner, path):
    import paper_2504_06182_gb300 as rr
    fx = json.load(open(path))
    grid = grid_from_rows(fx["grid"])
    m, n = grid.shape
    bird = fx.get("planner") == "bird"
    for layout in (rr.RR_U8, rr.RR_BITS32):
        host = grid if layout == rr.RR_U8 else gridgen.pack_bits32(grid).view(np.int32)
        g = torch.from_numpy(np.ascontiguousarray(host)).cuda()
        st, mv = planner.plan(g, tuple(fx["rect"]), layout=layout, n=n, bird=bird)
        assert st == fx["status"]
        assert mv.cpu().numpy().tolist() == fx["moves"]
    if fx["status"] == 0 and fx["moves"]:
        ops, mem = planner.batch(torch.tensor(fx["moves"], dtype=torch.int32).cuda(), m, n)
        assert ops.cpu().numpy().tolist() == fx["ops"]
        assert mem.cpu().numpy().tolist() == fx["members"]
