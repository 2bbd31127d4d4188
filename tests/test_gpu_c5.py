"""The served workload's grid sizes (sides 64..512, fill 0.6, centred target of
floor(0.7 * side)) through the batched entry point and through the server,
red-rec and bird, in both grid layouts: every status, move, batch and member
equals the oracle's (integers: exact). Sides above 256 take the 32-bit slot
links of the simulation and the largest shared-memory size classes."""
import numpy as np
import pytest

import gridgen
from tests.oracle_refs import path_steps, refs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

LARGE_SIDES = (288, 304, 336, 384, 432, 480, 512)


def _device_grid(grid, layout):
    from paper_2504_06182_gb300 import RR_U8
    if layout == RR_U8:
        return torch.from_numpy(np.ascontiguousarray(grid)).cuda()
    return torch.from_numpy(np.ascontiguousarray(gridgen.pack_bits32(grid).view(np.int32))).cuda()


def _expect_status(ref):
    import paper_2504_06182_gb300 as rr
    return rr.RR_OK if ref.status == 0 else rr.RR_INFEASIBLE


@pytest.mark.parametrize("bird", [False, True], ids=["redrec", "bird"])
def test_batched_served_sizes(bird):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2504_06182_gb300 as rr
    from paper_2504_06182_gb300.planner import Planner, pack_instances, unpack_instances

    insts = [gridgen.square_instance(61, g, s, 0.6) for g, s in enumerate(LARGE_SIDES + (64, 112, 200))]
    expect = refs([(i.grid, i.rect) for i in insts], bird=bird)
    assert all(e.status == 0 for e in expect[: len(LARGE_SIDES)])
    P = Planner(arena_bytes=8 << 30)
    try:
        entries, outs = [], []
        for g, (inst, e) in enumerate(zip(insts, expect)):
            s = inst.grid.shape[0]
            layout = rr.RR_BITS32 if g % 2 == 0 else rr.RR_U8
            k = max(len(e.moves), 1)
            steps = max(path_steps(e.moves), 1)
            mv = torch.empty((k, 4), dtype=torch.int32, device="cuda")
            ops = torch.empty((steps, 3), dtype=torch.int32, device="cuda")
            mem = torch.empty((steps,), dtype=torch.int32, device="cuda")
            entries.append(dict(grid=_device_grid(inst.grid, layout), layout=layout, m=s, n=s, rect=inst.rect,
                                moves=mv, cap_moves=k, ops=ops, cap_ops=steps, members=mem, cap_members=steps))
            outs.append((mv, ops, mem))
        dev = pack_instances(entries)
        flags = rr.RR_WITH_BATCH | (rr.RR_BIRD if bird else 0)
        assert rr.rr_plan_batched(P.ctx, dev, len(entries), 512, flags) == rr.RR_OK
        torch.cuda.synchronize()
        for g, (r, e, (mv, ops, mem)) in enumerate(zip(unpack_instances(dev, len(entries)), expect, outs)):
            assert r.status == _expect_status(e), (g, r.status, e.status)
            assert r.n_moves == len(e.moves), g
            if e.status != 0:
                continue
            assert (mv[: r.n_moves].cpu().numpy() == e.moves).all(), g
            assert r.n_ops == len(e.ops) and r.n_members == len(e.members), g
            assert (ops[: r.n_ops].cpu().numpy() == e.ops).all(), g
            assert (mem[: r.n_members].cpu().numpy() == e.members).all(), g
    finally:
        P.close()


@pytest.mark.parametrize("bird", [False, True], ids=["redrec", "bird"])
def test_server_served_sizes(bird):
    """Requests of the served stream's sizes (half of them above 256) admitted
    into overlapping waves: each result equals the oracle's plan and batches
    for that grid alone."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2504_06182_gb300 as rr
    from paper_2504_06182_gb300.planner import device_view

    insts = gridgen.mixed_instances(62, 10, sides=gridgen.SIDES_SERVED, p_lo=0.6, p_hi=0.6)
    insts += [gridgen.square_instance(63, g, s, 0.6) for g, s in enumerate(LARGE_SIDES[::2])]
    assert sum(i.grid.shape[0] > 256 for i in insts) >= 6
    expect = refs([(i.grid, i.rect) for i in insts], bird=bird)
    flags = rr.RR_WITH_BATCH | (rr.RR_BIRD if bird else 0)
    srv = rr.rr_serve_open(max_side=512, slots=8, streams=4, max_wave=3, flags=flags,
                           arena_bytes=2 << 30, heap_bytes=2 << 30)
    try:
        tickets = []
        for g, inst in enumerate(insts):
            m, n = inst.grid.shape
            if g % 2:
                st, t = rr.rr_serve_submit(srv, np.ascontiguousarray(inst.grid), rr.RR_U8, m, n, inst.rect)
            else:
                w = np.ascontiguousarray(gridgen.pack_bits32(inst.grid).view(np.int32))
                st, t = rr.rr_serve_submit(srv, w, rr.RR_BITS32, m, n, inst.rect)
            assert st == rr.RR_OK
            tickets.append(t)
        waited = 0
        for g, (inst, e, t) in enumerate(zip(insts, expect, tickets)):
            st, res = rr.rr_serve_poll(srv, t, timeout_us=300_000_000)
            assert st == rr.RR_OK, (g, st)
            assert res.status == _expect_status(e), (g, res.status, e.status)
            assert res.n_moves == len(e.moves), g
            if e.status == 0:
                assert (device_view(res.d_moves, (res.n_moves, 4)).cpu().numpy() == e.moves).all(), g
                assert res.n_ops == len(e.ops) and res.n_members == len(e.members), g
                assert (device_view(res.d_ops, (res.n_ops, 3)).cpu().numpy() == e.ops).all(), g
                assert (device_view(res.d_members, (res.n_members,)).cpu().numpy() == e.members).all(), g
            waited += res.t_admit_us > res.t_submit_us
            assert rr.rr_serve_release(srv, t) == rr.RR_OK
        assert waited > 0            # fewer slots than requests: later ones were admitted as slots freed
    finally:
        rr.rr_serve_close(srv)
