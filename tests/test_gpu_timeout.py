"""The failure path of the bounded device loops, without a fault: with the
iteration cap of rr_debug_guard_limit set low, the pairing loop (Alg. 1) and
the batching simulation (Alg. 4) stop and every entry point reports
RR_ERR_TIMEOUT (per instance in the batched call); with the cap removed, the
same context gives the oracle's results again."""
import numpy as np
import pytest

import gridgen
import oracle
from tests.oracle_refs import path_steps

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_capped_loops_report_timeout_and_the_context_recovers():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2504_06182_gb300 as rr
    from paper_2504_06182_gb300.planner import Planner, pack_instances, unpack_instances

    inst = gridgen.square_instance(0, 0, 32, 0.6, 20)
    ref = oracle.plan(inst.grid, inst.rect)
    rops, rmem = oracle.batch(ref.moves, 32, 32)
    assert ref.status == 0
    steps = path_steps(ref.moves)
    g = torch.from_numpy(inst.grid).cuda()
    mv_ref = torch.from_numpy(ref.moves).cuda()
    P = Planner(arena_bytes=256 << 20)
    try:
        assert rr.rr_debug_guard_limit(-1) == rr.RR_ERR_ARG
        assert rr.rr_debug_guard_limit(2) == rr.RR_OK
        out = torch.empty((len(ref.moves) + 1, 4), dtype=torch.int32, device="cuda")
        st, _ = rr.rr_plan(P.ctx, g, rr.RR_U8, 32, 32, inst.rect, out, len(ref.moves) + 1)
        assert st == rr.RR_ERR_TIMEOUT                        # the pairing loop ran out
        ops = torch.empty((steps, 3), dtype=torch.int32, device="cuda")
        mem = torch.empty((steps,), dtype=torch.int32, device="cuda")
        st, _, _ = rr.rr_batch(P.ctx, mv_ref, len(ref.moves), 32, 32, ops, steps, mem, steps)
        assert st == rr.RR_ERR_TIMEOUT                        # the simulation ran out
        st = rr.rr_plan_one(P.ctx, g, rr.RR_U8, 32, 32, inst.rect, rr.RR_WITH_BATCH, out, len(ref.moves) + 1,
                            ops, steps, mem, steps)[0]
        assert st == rr.RR_ERR_TIMEOUT
        e = dict(grid=g, layout=rr.RR_U8, m=32, n=32, rect=inst.rect, moves=out, cap_moves=len(ref.moves) + 1,
                 ops=ops, cap_ops=steps, members=mem, cap_members=steps)
        dev = pack_instances([e, e])
        assert rr.rr_plan_batched(P.ctx, dev, 2, 32, rr.RR_WITH_BATCH) == rr.RR_OK
        torch.cuda.synchronize()
        assert [x.status for x in unpack_instances(dev, 2)] == [rr.RR_ERR_TIMEOUT] * 2
        # a cap above what the loops need changes nothing
        assert rr.rr_debug_guard_limit(10 ** 9) == rr.RR_OK
        st, mv = P.plan(g, inst.rect)
        assert st == rr.RR_OK and (mv.cpu().numpy() == ref.moves).all()
    finally:
        assert rr.rr_debug_guard_limit(0) == rr.RR_OK
    try:
        # the built-in bounds again: the same context, the oracle's results
        st, mv = P.plan(g, inst.rect)
        assert st == rr.RR_OK and (mv.cpu().numpy() == ref.moves).all()
        o, m_ = P.batch(mv, 32, 32)
        assert (o.cpu().numpy() == rops).all() and (m_.cpu().numpy() == rmem).all()
        res = rr.rr_plan_one(P.ctx, g, rr.RR_U8, 32, 32, inst.rect, rr.RR_WITH_BATCH, out, len(ref.moves) + 1,
                             ops, steps, mem, steps)
        assert res[0] == rr.RR_OK and res[3] == len(rops)
        assert (ops[: len(rops)].cpu().numpy() == rops).all()
    finally:
        P.close()
