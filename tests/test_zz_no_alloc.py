"""rr_plan_noalloc: planning for callers that must not allocate device memory
(a real-time reconfiguration loop, where cudaMalloc can synchronise the device
and take unbounded time; work issued during graph capture; plug-ins whose
device memory belongs to another allocator). Its workspace is a fixed device
array, so its output must equal rr_plan's, call after call.

Collected last on purpose (file name): when it fails, a run that stops at the
first failure has already run every other test."""
import numpy as np
import pytest

import gridgen

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _device_grid(grid, layout):
    from paper_2504_06182_gb300 import RR_U8
    if layout == RR_U8:
        return torch.from_numpy(np.ascontiguousarray(grid)).cuda()
    return torch.from_numpy(np.ascontiguousarray(gridgen.pack_bits32(grid).view(np.int32))).cuda()


def test_noalloc_plan_equals_rr_plan_on_consecutive_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2504_06182_gb300 as rr
    from paper_2504_06182_gb300.planner import Planner

    cases = [(gridgen.square_instance(4, 0, 256, 0.6, 180), rr.RR_BITS32),
             (gridgen.square_instance(2, 0, 32, 0.6, 20), rr.RR_U8),
             (gridgen.square_instance(9, 1, 200, 0.55), rr.RR_U8)]
    P = Planner(arena_bytes=256 << 20)
    try:
        for inst, layout in cases:
            m, n = inst.grid.shape
            g = _device_grid(inst.grid, layout)
            st_ref, ref = P.plan(g, inst.rect, layout=layout, n=n)
            ref = ref.cpu().numpy()
            cap = max(len(ref), 1)
            out = torch.full((cap, 4), -1, dtype=torch.int32, device="cuda")
            st, k = rr.rr_plan_noalloc(g, layout, m, n, inst.rect, out, cap)
            assert st == st_ref, (st, st_ref)
            assert k == len(ref)
            assert (out[:k].cpu().numpy() == ref).all()
        # sizes beyond the fixed workspace are refused
        big = torch.zeros((300, 300), dtype=torch.uint8, device="cuda")
        st, _ = rr.rr_plan_noalloc(big, rr.RR_U8, 300, 300, (10, 10, 290, 290), out, cap)
        assert st == rr.RR_ERR_ARG
    finally:
        P.close()
