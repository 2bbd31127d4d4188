"""Serving (continuous batching): a burst of requests of mixed sizes is
admitted as slots free up and planned/batched in overlapping waves; every
result must equal the oracle's plan and batches of the same grid alone
(integer outputs: exact)."""
import numpy as np
import pytest

import gridgen
from tests.oracle_refs import refs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("max_wave", [5, 12])
def test_served_results_equal_alone(max_wave):
    """Waves of at most 5 run the simulation as one launch; waves of 12 fork
    it into size classes."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2504_06182_gb300 as rr

    insts = gridgen.mixed_instances(77, 40, sides=tuple(range(32, 257, 32)), p_lo=0.55, p_hi=0.7)
    expect = refs([(i.grid, i.rect) for i in insts])
    assert {e.status for e in expect} == {0, 1}
    srv = rr.rr_serve_open(max_side=256, slots=max(12, 2 * max_wave), streams=3, max_wave=max_wave,
                           flags=rr.RR_WITH_BATCH, arena_bytes=1 << 30, heap_bytes=1 << 30)
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
        overlapped = 0
        for e, t in zip(expect, tickets):
            st, res = rr.rr_serve_poll(srv, t, timeout_us=120_000_000)
            assert st == rr.RR_OK, st
            check_result(res, e)
            overlapped += res.t_admit_us > res.t_submit_us
            assert rr.rr_serve_release(srv, t) == rr.RR_OK
        # with fewer slots than the 40 requests submitted at once, later ones waited
        assert overlapped > 0
        # unknown ticket and oversize grids are refused
        assert rr.rr_serve_poll(srv, 10 ** 9)[0] == rr.RR_ERR_ARG
        big = np.zeros((300, 300), np.uint8)
        assert rr.rr_serve_submit(srv, big, rr.RR_U8, 300, 300, (1, 1, 299, 299))[0] == rr.RR_ERR_ARG
    finally:
        rr.rr_serve_close(srv)


def check_result(res, e):
    """A served result against the oracle's plan and batches of that grid."""
    import paper_2504_06182_gb300 as rr
    from paper_2504_06182_gb300.planner import device_view
    assert res.status == (rr.RR_OK if e.status == 0 else rr.RR_INFEASIBLE), (res.status, e.status)
    assert res.n_moves == len(e.moves)
    if e.status != 0:
        return
    assert (device_view(res.d_moves, (res.n_moves, 4)).cpu().numpy() == e.moves).all()
    assert res.n_ops == len(e.ops) and res.n_members == len(e.members)
    assert (device_view(res.d_ops, (res.n_ops, 3)).cpu().numpy() == e.ops).all()
    assert (device_view(res.d_members, (res.n_members,)).cpu().numpy() == e.members).all()


def test_served_admission_by_memory():
    """A small input pool (room for about three 256 x 256 requests) admits
    requests as their grid and move list fit: every result still equals
    the request planned alone, and a grid that could never fit is refused."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2504_06182_gb300 as rr

    insts = gridgen.mixed_instances(78, 24, sides=(32, 64, 128, 256), p_lo=0.6, p_hi=0.65)
    expect = refs([(i.grid, i.rect) for i in insts])
    per_max = 256 * 256 + 2 * 256 * 256 * 16           # grid bytes + move list of a 256 x 256 request
    srv = rr.rr_serve_open(max_side=512, slots=24, streams=4, max_wave=4, flags=rr.RR_WITH_BATCH,
                           arena_bytes=1 << 30, heap_bytes=1 << 30, input_bytes=3 * per_max + (1 << 20))
    try:
        big = np.zeros((512, 512), np.uint8)
        assert rr.rr_serve_submit(srv, big, rr.RR_U8, 512, 512, (1, 1, 511, 511))[0] == rr.RR_ERR_CAPACITY
        tickets = []
        for inst in insts:
            m, n = inst.grid.shape
            st, t = rr.rr_serve_submit(srv, np.ascontiguousarray(inst.grid), rr.RR_U8, m, n, inst.rect)
            assert st == rr.RR_OK
            tickets.append(t)
        for e, t in zip(expect, tickets):
            st, res = rr.rr_serve_poll(srv, t, timeout_us=120_000_000)
            assert st == rr.RR_OK, st
            check_result(res, e)
            assert rr.rr_serve_release(srv, t) == rr.RR_OK
    finally:
        rr.rr_serve_close(srv)
