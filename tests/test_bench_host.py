"""Host-side logic of bench.py (no GPU): the plain path's queueing model, the
traffic ratio read from the committed ncu record, the batched-transfer count,
the workload constructors, the per-rank seeds and the garbage-collector pause of
the timed loops."""
import hashlib
import json
import os

import numpy as np

import bench
import gridgen


def test_fifo_latencies_single_server():
    # arrivals at 0, 1, 2 with 2 s of service each: the server is busy from
    # 0 to 6, so the requests finish at 2, 4, 6
    assert bench.fifo_latencies([0.0, 1.0, 2.0], [2.0, 2.0, 2.0]) == [2.0, 3.0, 4.0]
    # an idle gap: the second request starts on arrival
    assert bench.fifo_latencies([0.0, 10.0], [1.0, 1.0]) == [1.0, 1.0]
    # Lindley's recursion against a direct restatement
    rng = np.random.default_rng(3)
    arr = np.cumsum(rng.exponential(1.0, 200))
    svc = rng.exponential(0.9, 200)
    lat = bench.fifo_latencies(arr, svc)
    wait = 0.0
    for i in range(200):
        if i:
            wait = max(0.0, wait + svc[i - 1] - (arr[i] - arr[i - 1]))
        assert abs(lat[i] - (wait + svc[i])) < 1e-9


def test_traffic_ratio_tracks_the_sources():
    """The ratio is reported only for the profiled kernel and only while the
    sources fingerprinted in the record are unchanged."""
    rec = json.load(open(bench.TRAFFIC_JSON))
    h = hashlib.sha256()
    for f in ("rr_batch.cuh", "rr_batch.cu", "rr_internal.cuh"):
        h.update(open(os.path.join(bench.ROOT, "paper_2504_06182_gb300", "csrc", f), "rb").read())
    expect = float(rec["ratio"]) if h.hexdigest()[:16] == rec["src_sha256_16"] else None
    assert bench.measured_traffic_ratio("k_sim") == expect
    assert bench.measured_traffic_ratio("k_bsort") is None
    assert bench.sources_fingerprint() == h.hexdigest()[:16]


def _fixture(name):
    return json.load(open(os.path.join(bench.ROOT, "tests", "golden", name + ".json")))


def test_nb_alpha_on_hand_worked_batches():
    """Batched transfers (Sec. V): batches holding some token's first step
    (one parallel extraction) plus batches holding some token's last step
    (one parallel implantation)."""
    # equal_exchange: batch 0 moves both tokens off their traps (one
    # extraction batch); move 0 ends in batch 1, move 1 in batch 2
    fx = _fixture("equal_exchange")
    assert bench.nb_alpha(fx["ops"], fx["members"]) == 1 + 2
    # many_to_one_redrec: both start in batch 0; move 0 ends in batch 1,
    # move 1 in batch 4
    fx = _fixture("many_to_one_redrec")
    assert bench.nb_alpha(fx["ops"], fx["members"]) == 1 + 2
    # the 2n chain: every batch holds one token, so no transfer is shared:
    # NB_alpha = N_alpha = 2 per move
    fx = _fixture("chain_2n")
    assert bench.nb_alpha(fx["ops"], fx["members"]) == 2 * len(fx["moves"])
    assert bench.nb_alpha(np.zeros((0, 3), np.int32), np.zeros(0, np.int32)) == 0


def test_served_requests_are_distinct_grids():
    a = [bench.served_grid(5, i) for i in range(6)]
    assert all(s in gridgen.SIDES_SERVED for _, _, s in a)
    assert len({(w.tobytes(), s) for w, _, s in a}) == 6
    w, rect, s = bench.served_grid(5, 3)
    assert rect == gridgen.centred_rect(s, s, int(0.7 * s), int(0.7 * s))
    assert (w == bench.served_grid(5, 3)[0]).all()


def test_paper_instances_are_the_paper_geometry_and_feasible():
    insts = bench.paper_instances()
    assert [i.grid.shape[1] for i in insts] == list(bench.PAPER_NTX)
    for i in insts:
        m, n = i.grid.shape
        assert m == (5 * n + 2) // 3
        assert i.rect == (i.rect[0], 0, i.rect[0] + n, n)
        assert int(i.grid.sum()) >= n * n


def test_rank_seeds_are_distinct_and_workloads_differ():
    seeds = [bench.rank_seed(0, r) for r in range(8)]
    assert len(set(seeds)) == 8
    a = gridgen.mixed_instances(seeds[0], 4)
    b = gridgen.mixed_instances(seeds[1], 4)
    assert any(x.grid.shape != y.grid.shape or (x.grid != y.grid).any() for x, y in zip(a, b))


def test_single_configs_match_the_named_sizes():
    names = [c[0] for c in bench.SINGLE_CONFIGS]
    sides = [c[1] for c in bench.SINGLE_CONFIGS]
    assert sides == [32, 256, 1024]
    for name, side, t, lay in bench.SINGLE_CONFIGS:
        assert f"{side}x{side}" in name and f"{t}x{t}" in name and lay in ("u8", "bits32")


def test_timed_region_pauses_the_garbage_collector():
    """Timed loops run with Python's cyclic collector off; it is back on
    afterwards, also when the loop raises."""
    import gc
    assert gc.isenabled()
    with bench.timed_region():
        assert not gc.isenabled()
    assert gc.isenabled()
    try:
        with bench.timed_region():
            raise RuntimeError("step failed")
    except RuntimeError:
        pass
    assert gc.isenabled()
    gc.disable()
    try:
        with bench.timed_region():
            assert not gc.isenabled()
        assert not gc.isenabled()      # a collector that was off stays off
    finally:
        gc.enable()

