"""The multi-GPU path of bench.py on CPU: two gloo ranks. Grids are
independent, so each rank plans its own workload (weak scaling) and the only
collectives are the barrier and the maximum of the ranks' times."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import gridgen
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        seed = bench.rank_seed(0, rank)
        insts = gridgen.mixed_instances(seed, 3)
        digest = [int(i.grid.sum()) * 1000 + i.grid.shape[0] for i in insts]
        same = [int(i.grid.sum()) * 1000 + i.grid.shape[0] for i in gridgen.mixed_instances(seed, 3)]
        mx = bench.max_over_ranks(1.5 + rank, "cpu", world)
        dist.barrier()
        out.put((rank, seed, digest, same, mx))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, d0, same0, m0), (r1, s1, d1, same1, m1) = res
    assert (r0, r1) == (0, 1) and s0 != s1
    assert d0 == same0 and d1 == same1          # each rank's workload is reproducible
    assert d0 != d1                              # and the ranks' workloads differ
    assert m0 == m1 == 2.5                       # both see the slowest rank's time
