"""rr_plan_noalloc: planning for callers that must not allocate device memory
(a real-time reconfiguration loop, where cudaMalloc can synchronise the
device and take unbounded time between imaging and the tweezer moves; a
plug-in whose device memory belongs to another allocator). Its workspace is
one fixed device array shared by every call, so each call must give the
oracle's plan (and rr_plan's) even though the previous call's contents are
still in that array.

Collected last on purpose (file name): when it fails, a run that stops at the
first failure has already run every other test."""
import numpy as np
import pytest

import gridgen
import oracle

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _device_grid(grid, layout):
    from paper_2504_06182_gb300 import RR_U8
    if layout == RR_U8:
        return torch.from_numpy(np.ascontiguousarray(grid)).cuda()
    return torch.from_numpy(np.ascontiguousarray(gridgen.pack_bits32(grid).view(np.int32))).cuda()


def _status(ref_status):
    import paper_2504_06182_gb300 as rr
    return rr.RR_OK if ref_status == 0 else rr.RR_INFEASIBLE


@pytest.mark.filterwarnings("ignore:The CUDA Graph is empty")
def test_noalloc_plan_equals_oracle_and_rr_plan_on_consecutive_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2504_06182_gb300 as rr
    from paper_2504_06182_gb300.planner import Planner

    full = np.ones((256, 256), np.uint8)
    full[:3, :] = 0                       # the whole grid as target, 768 holes: infeasible
    dense = (np.random.default_rng(3).random((256, 256)) < 0.995).astype(np.uint8)
    dense_rect = (0, 0, 250, 256)         # nearly the whole grid: the largest workspace demand
    cases = [(gridgen.square_instance(4, 0, 256, 0.6, 180).grid, gridgen.square_instance(4, 0, 256, 0.6, 180).rect,
              rr.RR_BITS32),
             (gridgen.square_instance(2, 0, 32, 0.6, 20).grid, gridgen.square_instance(2, 0, 32, 0.6, 20).rect,
              rr.RR_U8),
             (gridgen.square_instance(9, 1, 200, 0.55).grid, gridgen.square_instance(9, 1, 200, 0.55).rect, rr.RR_U8),
             (dense, dense_rect, rr.RR_U8),
             (full, (0, 0, 256, 256), rr.RR_BITS32),
             (dense, dense_rect, rr.RR_BITS32)]
    P = Planner(arena_bytes=256 << 20)
    try:
        for repeat in range(2):            # two calls in a row on every case
            for grid, rect, layout in cases:
                m, n = grid.shape
                ref = oracle.plan(grid, rect)
                g = _device_grid(grid, layout)
                st_ref, mv_ref = P.plan(g, rect, layout=layout, n=n)
                cap = max(len(ref.moves), 1)
                out = torch.full((cap, 4), -1, dtype=torch.int32, device="cuda")
                st, k = rr.rr_plan_noalloc(g, layout, m, n, rect, out, cap)
                assert st == _status(ref.status) == st_ref, (st, ref.status, st_ref)
                assert k == len(ref.moves) == len(mv_ref)
                got = out[:k].cpu().numpy()
                assert (got == ref.moves).all()
                assert (got == mv_ref.cpu().numpy()).all()
        # too little room: the required count comes back, nothing is written
        grid, rect, layout = cases[0]
        ref = oracle.plan(grid, rect)
        out = torch.full((1, 4), -7, dtype=torch.int32, device="cuda")
        st, k = rr.rr_plan_noalloc(_device_grid(grid, layout), layout, 256, 256, rect, out, 1)
        assert st == rr.RR_ERR_CAPACITY and k == len(ref.moves)
        assert (out.cpu() == -7).all()
        # sizes beyond the fixed workspace are refused
        big = torch.zeros((300, 300), dtype=torch.uint8, device="cuda")
        st, _ = rr.rr_plan_noalloc(big, rr.RR_U8, 300, 300, (10, 10, 290, 290), out, 1)
        assert st == rr.RR_ERR_ARG
        # a capturing stream is refused before anything is enqueued
        s = torch.cuda.Stream()
        gr = torch.cuda.CUDAGraph()
        g = _device_grid(cases[1][0], rr.RR_U8)
        torch.cuda.synchronize()
        with torch.cuda.graph(gr, stream=s):
            st, _ = rr.rr_plan_noalloc(g, rr.RR_U8, 32, 32, cases[1][1], out, 1, stream=s)
        assert st == rr.RR_ERR_ARG
    finally:
        P.close()
