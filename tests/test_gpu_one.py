"""rr_plan_one (one grid planned and batched by one kernel launch) against the
oracle, element by element: random small rectangles in both layouts, the
32 x 32 and 256 x 256 workloads, red-rec and bird, both readings of target
sub-rectangles, infeasible grids, and the capacity protocol; every call is a
single launch."""
import numpy as np
import pytest

import gridgen
import oracle
from tests.oracle_refs import path_steps

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2504_06182_gb300 as rr
    c = rr.rr_ctx_create(1 << 30)
    yield c
    rr.rr_ctx_destroy(c)


def _device_grid(grid, layout):
    from paper_2504_06182_gb300 import RR_U8
    if layout == RR_U8:
        return torch.from_numpy(np.ascontiguousarray(grid)).cuda()
    return torch.from_numpy(np.ascontiguousarray(gridgen.pack_bits32(grid).view(np.int32))).cuda()


def run_one(ctx, grid, rect, layout, bird=False, strict=False, batch=True, caps=(1, 1)):
    """caps: room for moves and for batches (ops and members)."""
    import paper_2504_06182_gb300 as rr
    m, n = grid.shape
    k_cap, s_cap = caps
    mv = torch.full((max(k_cap, 1), 4), -1, dtype=torch.int32, device="cuda")
    ops = torch.full((max(s_cap, 1), 3), -1, dtype=torch.int32, device="cuda")
    mem = torch.full((max(s_cap, 1),), -1, dtype=torch.int32, device="cuda")
    flags = (rr.RR_WITH_BATCH if batch else 0) | (rr.RR_BIRD if bird else 0) | (rr.RR_STRICT_RESERVOIR if strict else 0)
    n0 = rr.rr_launch_count(ctx)
    st, nm, ns, no, nmem = rr.rr_plan_one(ctx, _device_grid(grid, layout), layout, m, n, rect, flags, mv, k_cap,
                                          ops, s_cap, mem, s_cap)
    assert rr.rr_launch_count(ctx) - n0 == 1
    return st, nm, ns, no, nmem, mv, ops, mem


def check(ctx, grid, rect, layout, bird=False, strict=False, batch=True):
    import paper_2504_06182_gb300 as rr
    ref = (oracle.bird if bird else oracle.plan)(grid, rect, strict=strict)
    caps = (len(ref.moves) + 1, path_steps(ref.moves) + 1)
    st, nm, ns, no, nmem, mv, ops, mem = run_one(ctx, grid, rect, layout, bird, strict, batch, caps)
    assert st == (rr.RR_OK if ref.status == 0 else rr.RR_INFEASIBLE), (st, ref.status, grid.shape, rect)
    assert nm == len(ref.moves)
    if ref.status != 0:
        return ref
    assert (mv[:nm].cpu().numpy() == ref.moves).all()
    assert ns == path_steps(ref.moves)
    if batch:
        rops, rmem = oracle.batch(ref.moves, *grid.shape)
        assert no == len(rops) and nmem == len(rmem)
        assert (ops[:no].cpu().numpy() == rops).all()
        assert (mem[:nmem].cpu().numpy() == rmem).all()
    return ref


def test_one_random_small_grids(ctx):
    import paper_2504_06182_gb300 as rr
    rng = np.random.default_rng(2468)
    feasible = 0
    for trial in range(240):
        m, n = int(rng.integers(1, 70)), int(rng.integers(1, 70))
        grid = (rng.random((m, n)) < rng.uniform(0.3, 0.95)).astype(np.uint8)
        h, w = int(rng.integers(1, m + 1)), int(rng.integers(1, n + 1))
        r0, c0 = int(rng.integers(0, m - h + 1)), int(rng.integers(0, n - w + 1))
        ref = check(ctx, grid, (r0, c0, r0 + h, c0 + w), rr.RR_U8 if trial % 2 else rr.RR_BITS32,
                    bird=trial % 3 == 1, strict=trial % 7 == 3, batch=trial % 5 != 4)
        feasible += ref.status == 0
    assert feasible > 80


@pytest.mark.parametrize("seed", range(6))
def test_one_grid_32(ctx, seed):
    import paper_2504_06182_gb300 as rr
    inst = gridgen.square_instance(seed, 0, 32, 0.6, 20)
    check(ctx, inst.grid, inst.rect, rr.RR_U8)
    check(ctx, inst.grid, inst.rect, rr.RR_BITS32, bird=True)


@pytest.mark.parametrize("bird", [False, True], ids=["redrec", "bird"])
def test_one_grid_256(ctx, bird):
    import paper_2504_06182_gb300 as rr
    inst = gridgen.square_instance(1, 0, 256, 0.6, 180)
    ref = check(ctx, inst.grid, inst.rect, rr.RR_BITS32, bird=bird)
    assert ref.status == 0


def test_one_paper_geometry_and_edges(ctx):
    import paper_2504_06182_gb300 as rr
    for n_tx in (32, 64, 150):
        inst = gridgen.paper_instance(42, 0, n_tx)
        check(ctx, inst.grid, inst.rect, rr.RR_BITS32)
    check(ctx, np.zeros((8, 8), np.uint8), (2, 2, 6, 6), rr.RR_U8)                 # no atoms: infeasible
    check(ctx, np.ones((5, 7), np.uint8), (0, 0, 5, 7), rr.RR_U8)                  # target = whole grid, 0 moves
    check(ctx, np.ones((1, 1), np.uint8), (0, 0, 1, 1), rr.RR_BITS32)
    chain = np.zeros((64, 1), np.uint8)
    chain[:32] = 1
    check(ctx, chain, (32, 0, 64, 1), rr.RR_U8)                                    # the 2n chain


def test_one_capacity_and_arguments(ctx):
    import paper_2504_06182_gb300 as rr
    inst = gridgen.square_instance(3, 0, 48, 0.6)
    ref = oracle.plan(inst.grid, inst.rect)
    steps = path_steps(ref.moves)
    st, nm, *_ = run_one(ctx, inst.grid, inst.rect, rr.RR_U8, caps=(3, steps))
    assert st == rr.RR_ERR_CAPACITY and nm == len(ref.moves)
    st, nm, ns, no, nmem, *_ = run_one(ctx, inst.grid, inst.rect, rr.RR_U8, caps=(len(ref.moves), 5))
    assert st == rr.RR_ERR_CAPACITY and nm == len(ref.moves) and nmem == steps and no >= 5
    g = _device_grid(inst.grid, rr.RR_U8)
    out = torch.empty((4, 4), dtype=torch.int32, device="cuda")
    big = torch.zeros((300, 300), dtype=torch.uint8, device="cuda")
    assert rr.rr_plan_one(ctx, big, rr.RR_U8, 300, 300, (10, 10, 290, 290), 0, out, 4)[0] == rr.RR_ERR_ARG
    assert rr.rr_plan_one(ctx, g, rr.RR_U8, 48, 48, (0, 0, 60, 48), 0, out, 4)[0] == rr.RR_ERR_ARG
    assert rr.rr_plan_one(ctx, g, rr.RR_U8, 48, 48, inst.rect, 1 << 9, out, 4)[0] == rr.RR_ERR_ARG
    # the context stays usable: a full call after the refusals
    check(ctx, inst.grid, inst.rect, rr.RR_U8)


@pytest.mark.parametrize("n", [64, 65, 70])
def test_one_ready_set_beyond_registers(ctx, n):
    """Every column starts with a ready move (4 atoms over 4 band rows, full
    width): n moves ready at once. Up to 64 the simulation keeps them in
    registers; beyond, the general simulation takes over; the batches are
    the oracle's either way."""
    import paper_2504_06182_gb300 as rr
    grid = np.zeros((8, n), np.uint8)
    grid[:4] = 1
    ref = check(ctx, grid, (4, 0, 8, n), rr.RR_U8)
    assert ref.status == 0 and len(ref.moves) == 4 * n
