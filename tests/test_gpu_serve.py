"""Serving (continuous batching): a burst of requests of mixed sizes is
admitted as slots free up and planned/batched in overlapping waves; every
result must equal the same request planned and batched alone (integer
outputs: exact)."""
import numpy as np
import pytest

import gridgen

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("max_wave", [5, 12])
def test_served_results_equal_alone(max_wave):
    """Waves of at most 5 run the simulation as one launch; waves of 12 fork
    it into size classes."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2504_06182_gb300 as rr
    from paper_2504_06182_gb300.planner import Planner, device_view

    insts = gridgen.mixed_instances(77, 40, sides=tuple(range(32, 257, 32)), p_lo=0.55, p_hi=0.7)
    srv = rr.rr_serve_open(max_side=256, slots=max(12, 2 * max_wave), streams=3, max_wave=max_wave,
                           flags=rr.RR_WITH_BATCH, arena_bytes=1 << 30, heap_bytes=1 << 30)
    P = Planner(arena_bytes=1 << 30)
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
        for inst, t in zip(insts, tickets):
            st, res = rr.rr_serve_poll(srv, t, timeout_us=120_000_000)
            assert st == rr.RR_OK, st
            m, n = inst.grid.shape
            st_ref, mv_ref = P.plan(torch.from_numpy(inst.grid).cuda(), inst.rect, layout=rr.RR_U8, n=n)
            assert res.status == st_ref
            assert res.n_moves == len(mv_ref)
            mv = device_view(res.d_moves, (res.n_moves, 4))
            assert torch.equal(mv, mv_ref)
            if st_ref == rr.RR_OK and len(mv_ref):
                ops_ref, mem_ref = P.batch(mv_ref, m, n)
                assert res.n_ops == len(ops_ref) and res.n_members == len(mem_ref)
                assert torch.equal(device_view(res.d_ops, (res.n_ops, 3)), ops_ref)
                assert torch.equal(device_view(res.d_members, (res.n_members,)), mem_ref)
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
        P.close()


def test_served_admission_by_memory():
    """A small input pool (room for about three 256 x 256 requests) admits
    requests as their grid and move list fit: every result still equals
    the request planned alone, and a grid that could never fit is refused."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2504_06182_gb300 as rr
    from paper_2504_06182_gb300.planner import Planner, device_view

    insts = gridgen.mixed_instances(78, 24, sides=(32, 64, 128, 256), p_lo=0.6, p_hi=0.65)
    per_max = 256 * 256 + 2 * 256 * 256 * 16           # grid bytes + move list of a 256 x 256 request
    srv = rr.rr_serve_open(max_side=512, slots=24, streams=4, max_wave=4, flags=rr.RR_WITH_BATCH,
                           arena_bytes=1 << 30, heap_bytes=1 << 30, input_bytes=3 * per_max + (1 << 20))
    P = Planner(arena_bytes=1 << 30)
    try:
        big = np.zeros((512, 512), np.uint8)
        assert rr.rr_serve_submit(srv, big, rr.RR_U8, 512, 512, (1, 1, 511, 511))[0] == rr.RR_ERR_CAPACITY
        tickets = []
        for inst in insts:
            m, n = inst.grid.shape
            st, t = rr.rr_serve_submit(srv, np.ascontiguousarray(inst.grid), rr.RR_U8, m, n, inst.rect)
            assert st == rr.RR_OK
            tickets.append(t)
        for inst, t in zip(insts, tickets):
            st, res = rr.rr_serve_poll(srv, t, timeout_us=120_000_000)
            assert st == rr.RR_OK, st
            m, n = inst.grid.shape
            st_ref, mv_ref = P.plan(torch.from_numpy(inst.grid).cuda(), inst.rect, layout=rr.RR_U8, n=n)
            assert res.status == st_ref and res.n_moves == len(mv_ref)
            assert torch.equal(device_view(res.d_moves, (res.n_moves, 4)), mv_ref)
            if st_ref == rr.RR_OK and len(mv_ref):
                ops_ref, mem_ref = P.batch(mv_ref, m, n)
                assert torch.equal(device_view(res.d_ops, (res.n_ops, 3)), ops_ref)
                assert torch.equal(device_view(res.d_members, (res.n_members,)), mem_ref)
            assert rr.rr_serve_release(srv, t) == rr.RR_OK
    finally:
        rr.rr_serve_close(srv)
        P.close()
