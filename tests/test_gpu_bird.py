"""The bird planner (Alg. 2, Sec. III.E) on the GPU against the oracle,
element by element (bit-exact), through the C ABI: single grids in both
layouts from tiny random rectangles to 256 x 256, the paper's runtime
geometry, mixed 32..256 grids through the batched entry point (planning and
batching, pipelined), and a 1024 x 1024 grid checked by replay."""
import numpy as np
import pytest

import gridgen
import oracle
from tests.checks import replay_moves, assert_target_full

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def planner():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_06182_gb300.planner import Planner
    p = Planner(arena_bytes=4 << 30)
    yield p
    p.close()


def to_device(grid, layout):
    from paper_2504_06182_gb300 import RR_U8
    if layout == RR_U8:
        return torch.from_numpy(np.ascontiguousarray(grid)).cuda()
    words = gridgen.pack_bits32(grid).view(np.int32)
    return torch.from_numpy(np.ascontiguousarray(words)).cuda()


def check_bird(planner, grid, rect, layout, with_batch=True):
    ref = oracle.bird(grid, rect)
    m, n = grid.shape
    st, mv = planner.plan(to_device(grid, layout), rect, layout=layout, n=n, bird=True)
    mv = mv.cpu().numpy()
    assert st == ref.status, (st, ref.status, grid.shape, rect)
    assert mv.shape == ref.moves.shape, (mv.shape, ref.moves.shape)
    if len(mv):
        bad = np.nonzero((mv != ref.moves).any(axis=1))[0]
        assert len(bad) == 0, f"first mismatch at move {bad[0]}: gpu {mv[bad[0]]} oracle {ref.moves[bad[0]]}"
    if with_batch and ref.status == 0:
        rops, rmem = oracle.batch(ref.moves, m, n)
        ops, mem = planner.batch(torch.from_numpy(ref.moves).cuda(), m, n)
        assert (ops.cpu().numpy() == rops).all() and ops.shape[0] == len(rops)
        assert (mem.cpu().numpy() == rmem).all() and mem.shape[0] == len(rmem)
    return ref


def random_case(rng):
    m = int(rng.integers(1, 70))
    n = int(rng.integers(1, 70))
    grid = (rng.random((m, n)) < rng.uniform(0.2, 0.95)).astype(np.uint8)
    h = int(rng.integers(1, m + 1))
    r0 = int(rng.integers(0, m - h + 1))
    w = int(rng.integers(1, n + 1))
    c0 = int(rng.integers(0, n - w + 1))
    return grid, (r0, c0, r0 + h, c0 + w)


def test_bird_random_small_grids(planner):
    from paper_2504_06182_gb300 import RR_BITS32, RR_U8
    rng = np.random.default_rng(4321)
    feasible = with_recv = 0
    for trial in range(400):
        grid, rect = random_case(rng)
        ref = check_bird(planner, grid, rect, RR_U8 if trial % 2 else RR_BITS32, with_batch=trial % 4 == 0)
        feasible += ref.status == 0
        r0, c0, r1, c1 = rect
        with_recv += ref.status == 0 and any(grid[:, c].sum() < r1 - r0 for c in range(c0, c1))
    assert feasible > 100 and with_recv > 50


@pytest.mark.parametrize("seed", range(10))
def test_bird_grid_32(planner, seed):
    from paper_2504_06182_gb300 import RR_U8
    inst = gridgen.square_instance(seed, 0, 32, 0.6, 20)
    check_bird(planner, inst.grid, inst.rect, RR_U8)


@pytest.mark.parametrize("seed", range(3))
def test_bird_grid_256(planner, seed):
    from paper_2504_06182_gb300 import RR_BITS32
    inst = gridgen.square_instance(seed, 0, 256, 0.6, 180)
    ref = check_bird(planner, inst.grid, inst.rect, RR_BITS32, with_batch=seed == 0)
    assert ref.status == 0


@pytest.mark.parametrize("n_tx", [32, 64, 128, 256])
def test_bird_paper_geometry(planner, n_tx):
    """The paper's runtime geometry (full-width target of n_tx rows in
    ceil(n_tx / 0.6) rows): a feasible and an infeasible instance. Atoms
    barely outnumber targets here, so the last columns find their tokens far
    away in nearly empty reservoirs (the kernel's counting search)."""
    from paper_2504_06182_gb300 import RR_BITS32, RR_U8
    seen = set()
    for g in range(40):
        inst = gridgen.paper_instance(41, g, n_tx)
        ref = oracle.bird(inst.grid, inst.rect)
        if ref.status in seen:
            continue
        seen.add(ref.status)
        check_bird(planner, inst.grid, inst.rect, RR_U8)
        check_bird(planner, inst.grid, inst.rect, RR_BITS32, with_batch=False)
        if len(seen) == 2:
            break
    assert seen == {0, 1}


@pytest.mark.parametrize("count", [48, 300])
def test_bird_batched_mixed(planner, count):
    """Mixed 32..256 grids through rr_plan_batched with RR_BIRD and batching
    (300 grids run pipelined by size), each grid against the oracle."""
    import paper_2504_06182_gb300 as rr
    from paper_2504_06182_gb300.planner import pack_instances, plan_batched, unpack_instances
    insts = gridgen.mixed_instances(17, count)
    refs = [oracle.bird(i.grid, i.rect) for i in insts]
    entries, outs = [], []
    for inst, ref in zip(insts, refs):
        s = inst.grid.shape[0]
        k = max(len(ref.moves), 1)
        mvs = ref.moves
        steps = int((np.abs(mvs[:, 0] - mvs[:, 2]) + np.abs(mvs[:, 1] - mvs[:, 3])).sum()) if len(mvs) else 0
        mv = torch.empty((k, 4), dtype=torch.int32, device="cuda")
        ops = torch.empty((max(steps, 1), 3), dtype=torch.int32, device="cuda")
        mem = torch.empty((max(steps, 1),), dtype=torch.int32, device="cuda")
        entries.append(dict(grid=to_device(inst.grid, rr.RR_BITS32), layout=rr.RR_BITS32, m=s, n=s, rect=inst.rect,
                            moves=mv, cap_moves=k, ops=ops, cap_ops=max(steps, 1), members=mem,
                            cap_members=max(steps, 1)))
        outs.append((mv, ops, mem))
    dev = pack_instances(entries)
    plan_batched(planner, dev, len(entries), 256, with_batch=True, bird=True)
    torch.cuda.synchronize()
    res = unpack_instances(dev, len(entries))
    nbatched = 0
    for inst, ref, r, (mv, ops, mem) in zip(insts, refs, res, outs):
        assert r.status == (rr.RR_OK if ref.status == 0 else rr.RR_INFEASIBLE), r.status
        assert r.n_moves == len(ref.moves)
        if ref.status != 0:
            continue
        assert (mv[: r.n_moves].cpu().numpy() == ref.moves).all()
        if nbatched < 60:
            rops, rmem = oracle.batch(ref.moves, *inst.grid.shape)
            assert r.n_ops == len(rops) and r.n_members == len(rmem)
            assert (ops[: r.n_ops].cpu().numpy() == rops).all()
            assert (mem[: r.n_members].cpu().numpy() == rmem).all()
            nbatched += 1
    assert nbatched > 10


def test_bird_capacity_and_infeasible(planner):
    import paper_2504_06182_gb300 as rr
    inst = gridgen.square_instance(3, 0, 64, 0.6, 44)
    ref = oracle.bird(inst.grid, inst.rect)
    assert ref.status == 0 and len(ref.moves) > 10
    g = to_device(inst.grid, rr.RR_U8)
    small = torch.empty((5, 4), dtype=torch.int32, device="cuda")
    st, k = rr.rr_bird_plan(planner.ctx, g, rr.RR_U8, 64, 64, inst.rect, small, 5)
    assert st == rr.RR_ERR_CAPACITY and k == len(ref.moves)
    empty = torch.zeros((16, 16), dtype=torch.uint8, device="cuda")
    st, k = rr.rr_bird_plan(planner.ctx, empty, rr.RR_U8, 16, 16, (4, 4, 12, 12), small, 5)
    assert st == rr.RR_INFEASIBLE and k == 0


def test_bird_grid_1024_replay(planner):
    """Full-size 1024 x 1024 grid with a centred 720 x 720 target (too large
    for the oracle's literal window scan over the whole plan): the GPU's bird
    plan equals the oracle's for the column phase and the first eight
    receiver units (the oracle stopped there), starts with red-rec's column
    phase, replays without obstruction and fills the target."""
    from paper_2504_06182_gb300 import RR_BITS32
    inst = gridgen.square_instance(0, 0, 1024, 0.6, 720)
    g = to_device(inst.grid, RR_BITS32)
    st, mv = planner.plan(g, inst.rect, layout=RR_BITS32, n=1024, bird=True)
    st2, rmv = planner.plan(g, inst.rect, layout=RR_BITS32, n=1024)
    assert st == st2 == 0
    mv, rmv = mv.cpu().numpy(), rmv.cpu().numpy()
    # the column phase: every move before the first one into a receiver
    # (a target column with fewer atoms than target rows)
    r0, c0, r1, c1 = inst.rect
    recv = np.zeros(1024, dtype=bool)
    recv[c0:c1] = inst.grid[:, c0:c1].sum(axis=0) < r1 - r0
    ncol = int(np.argmax(recv[mv[:, 3]]))
    assert ncol > 0 and ncol == int(np.argmax(recv[rmv[:, 3]]))
    assert (mv[:ncol] == rmv[:ncol]).all()
    pref = oracle.bird_prefix(inst.grid, inst.rect, 8)
    assert len(pref.moves) > ncol
    assert (mv[: len(pref.moves)] == pref.moves).all()
    final = replay_moves(inst.grid, inst.rect, mv)
    assert_target_full(final, inst.rect, inst.grid)


def test_bird_grid_1024_full_digest(planner):
    """The same 1024 x 1024 grid: the GPU's complete bird plan and all of its
    batches (85.7 M of them) against the SHA-256 digests of the oracle's
    complete outputs (tests/golden/digests/oracle_1024.json, written by
    tests/golden/digests/make_digests.py from the oracle alone)."""
    import hashlib
    import json
    import os
    from paper_2504_06182_gb300 import RR_BITS32

    def sha(a):
        return hashlib.sha256(np.ascontiguousarray(a, dtype="<i4").tobytes()).hexdigest()
    with open(os.path.join(os.path.dirname(__file__), "golden", "digests", "oracle_1024.json")) as f:
        gold = json.load(f)["bird"]
    inst = gridgen.square_instance(0, 0, 1024, 0.6, 720)
    st, mv = planner.plan(to_device(inst.grid, RR_BITS32), inst.rect, layout=RR_BITS32, n=1024, bird=True)
    assert st == gold["status"] == 0
    assert len(mv) == gold["n_moves"] and sha(mv.cpu().numpy()) == gold["moves_sha256"]
    ops, mem = planner.batch(mv, 1024, 1024)
    assert len(ops) == gold["n_ops"] and len(mem) == gold["n_members"]
    assert sha(ops.cpu().numpy()) == gold["ops_sha256"]
    assert sha(mem.cpu().numpy()) == gold["members_sha256"]


def test_bird_served():
    """Served requests with RR_BIRD (waves of at most 5, three streams):
    every result equals the oracle's bird plan and its batches."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2504_06182_gb300 as rr
    from paper_2504_06182_gb300.planner import device_view
    insts = gridgen.mixed_instances(78, 24, sides=tuple(range(32, 161, 32)), p_lo=0.55, p_hi=0.7)
    srv = rr.rr_serve_open(max_side=256, slots=10, streams=3, max_wave=5, flags=rr.RR_WITH_BATCH | rr.RR_BIRD,
                           arena_bytes=1 << 30, heap_bytes=1 << 30)
    try:
        tickets = []
        for inst in insts:
            m, n = inst.grid.shape
            st, t = rr.rr_serve_submit(srv, np.ascontiguousarray(inst.grid), rr.RR_U8, m, n, inst.rect)
            assert st == rr.RR_OK
            tickets.append(t)
        for inst, t in zip(insts, tickets):
            st, res = rr.rr_serve_poll(srv, t, timeout_us=120_000_000)
            assert st == rr.RR_OK, st
            ref = oracle.bird(inst.grid, inst.rect)
            assert res.status == ref.status and res.n_moves == len(ref.moves)
            if ref.status == 0:
                assert (device_view(res.d_moves, (res.n_moves, 4)).cpu().numpy() == ref.moves).all()
                rops, rmem = oracle.batch(ref.moves, *inst.grid.shape)
                assert res.n_ops == len(rops) and res.n_members == len(rmem)
                assert (device_view(res.d_ops, (res.n_ops, 3)).cpu().numpy() == rops).all()
                assert (device_view(res.d_members, (res.n_members,)).cpu().numpy() == rmem).all()
            assert rr.rr_serve_release(srv, t) == rr.RR_OK
    finally:
        rr.rr_serve_close(srv)


@pytest.mark.parametrize("bird", [False, True])
def test_strict_reservoir_mode(planner, bird):
    """RR_STRICT_RESERVOIR (outer columns donate only their reservoir-row
    atoms) for red-rec and bird: random rectangles, both layouts, plans equal
    the oracle's strict plans; batched calls with the flag too."""
    import paper_2504_06182_gb300 as rr
    from paper_2504_06182_gb300.planner import pack_instances, plan_batched, unpack_instances
    rng = np.random.default_rng(99)
    f = oracle.bird if bird else oracle.plan
    feasible = 0
    cases = [random_case(rng) for _ in range(200)]
    for t, (grid, rect) in enumerate(cases):
        ref = f(grid, rect, strict=True)
        m, n = grid.shape
        layout = rr.RR_U8 if t % 2 else rr.RR_BITS32
        st, mv = planner.plan(to_device(grid, layout), rect, layout=layout, n=n, bird=bird, strict=True)
        assert st == ref.status, (t, st, ref.status)
        assert (mv.cpu().numpy() == ref.moves).all() and mv.shape[0] == len(ref.moves)
        feasible += ref.status == 0
    assert feasible > 50
    # batched, with batching
    entries, outs, refs = [], [], []
    for grid, rect in cases[:40]:
        ref = f(grid, rect, strict=True)
        m, n = grid.shape
        k = max(len(ref.moves), 1)
        steps = int((np.abs(ref.moves[:, 0] - ref.moves[:, 2]) + np.abs(ref.moves[:, 1] - ref.moves[:, 3])).sum()) \
            if len(ref.moves) else 0
        mv = torch.empty((k, 4), dtype=torch.int32, device="cuda")
        ops = torch.empty((max(steps, 1), 3), dtype=torch.int32, device="cuda")
        mem = torch.empty((max(steps, 1),), dtype=torch.int32, device="cuda")
        entries.append(dict(grid=to_device(grid, rr.RR_U8), layout=rr.RR_U8, m=m, n=n, rect=rect, moves=mv,
                            cap_moves=k, ops=ops, cap_ops=max(steps, 1), members=mem, cap_members=max(steps, 1)))
        outs.append((mv, ops, mem))
        refs.append((grid, ref))
    dev = pack_instances(entries)
    plan_batched(planner, dev, len(entries), 70, with_batch=True, bird=bird, strict=True)
    torch.cuda.synchronize()
    for (grid, ref), r, (mv, ops, mem) in zip(refs, unpack_instances(dev, len(entries)), outs):
        assert r.status == (rr.RR_OK if ref.status == 0 else rr.RR_INFEASIBLE)
        assert r.n_moves == len(ref.moves)
        if ref.status == 0:
            assert (mv[: r.n_moves].cpu().numpy() == ref.moves).all()
            rops, rmem = oracle.batch(ref.moves, *grid.shape)
            assert r.n_ops == len(rops) and (ops[: r.n_ops].cpu().numpy() == rops).all()
            assert r.n_members == len(rmem) and (mem[: r.n_members].cpu().numpy() == rmem).all()


def test_bird_edge_cases(planner):
    """Adversarial shapes for bird (and its strict mode): no atoms, a full
    grid, a target covering the grid, h = m, 1 x 1, one column, one row, every
    column at zero surplus, ragged 32-tiles."""
    import paper_2504_06182_gb300 as rr
    rng = np.random.default_rng(8)
    cases = [(np.zeros((8, 8), np.uint8), (2, 2, 6, 6)),
             (np.ones((8, 8), np.uint8), (2, 2, 6, 6)),
             (np.ones((5, 7), np.uint8), (0, 0, 5, 7)),
             (np.ones((1, 1), np.uint8), (0, 0, 1, 1)),
             ((rng.random((97, 1)) < 0.6).astype(np.uint8), (30, 0, 60, 1)),
             ((rng.random((1, 97)) < 0.9).astype(np.uint8), (0, 3, 1, 90)),
             ((rng.random((65, 65)) < 0.6).astype(np.uint8), (10, 10, 55, 55))]
    g = np.ones((6, 4), np.uint8); g[3, 1] = 0
    cases.append((g, (0, 1, 6, 3)))                                   # h = m, one hole
    z = np.zeros((12, 9), np.uint8)
    for c in range(9):                                                # 4 atoms per column, rows vary
        z[rng.choice(12, 4, replace=False), c] = 1
    cases.append((z, (4, 0, 8, 9)))                                   # every column at zero surplus
    for i, (grid, rect) in enumerate(cases):
        m, n = grid.shape
        layout = rr.RR_U8 if i % 2 else rr.RR_BITS32
        for strict in (False, True):
            ref = oracle.bird(grid, rect, strict=strict)
            st, mv = planner.plan(to_device(grid, layout), rect, layout=layout, n=n, bird=True, strict=strict)
            assert st == ref.status, (i, strict, st, ref.status)
            assert mv.cpu().numpy().tolist() == ref.moves.tolist(), (i, strict)
