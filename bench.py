#!/usr/bin/env python
"""Benchmark of the red-rec planning + batching path on one GB300.

Workload (one step): 4096 independent square grids, side uniform over
{32, 48, ..., 256}, fill p uniform in [0.5, 0.7], centred target of side
floor(0.7 * side), bit-packed uint32 rows; the whole batch is planned
(Alg. 1) and batched (Alg. 4) by one rr_plan_batched(RR_WITH_BATCH) call.
Inputs are seeded synthetic grids (gridgen), resident in HBM before timing.

The line also carries, measured after the timed steps: the same grids
replayed from a captured CUDA graph and end to end with host copies; the
plain one-grid-per-call path; the paper's runtime geometry (red-rec and bird
plans against the single-thread oracle); the served stream; and the bird
planner (Alg. 2) with batching on the same grids (`bird`, with its own CPU
oracle sample).

`--impl reference` times the CPU oracle instead (bounded samples of the same
workload on the host cores). Under torchrun every rank plans its own 4096
grids (weak scaling); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import contextlib
import gc
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import gridgen  # noqa: E402

# The served run keeps dozens of streams busy; the device's default of 8
# hardware work queues would make them wait on one another (set before CUDA
# initialises; it lasts for this process only).
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

@contextlib.contextmanager
def timed_region():
    """Timed loops run with Python's cyclic garbage collector paused (after a
    collection), so that a collection pass over the many small host objects of
    the workload (descriptors, per-grid records) cannot stall the host between
    kernel launches of a timed step."""
    gc.collect()
    was = gc.isenabled()
    gc.disable()
    try:
        yield
    finally:
        if was:
            gc.enable()


METRIC = "red-rec grids/s and p50/p99 plan latency, batched/served vs plain; %HBM roof"
WORKLOAD = "4096 square grids, side U{32..256 step 16}, p U[0.5,0.7], centred floor(0.7*side) target, bits32"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--count", type=int, default=4096)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--cpu-budget", type=float, default=15.0, help="seconds of oracle work for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--plain-sample", type=int, default=96, help="grids run one per call for the plain baseline")
    ap.add_argument("--served-requests", type=int, default=1000,
                    help="requests of the served high-load run (0: skip the served runs)")
    ap.add_argument("--served-load", type=float, default=0.8, help="arrival rate as a fraction of saturation")
    ap.add_argument("--served-plain-requests", type=int, default=48,
                    help="requests per arrival rate at fractions of the plain path's rate")
    ap.add_argument("--no-bird", action="store_true", help="skip the bird planner's line")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the library's default launch configuration (for profiling fixed launches)")
    ap.add_argument("--configs", action="store_true",
                    help="instead of the bench line: one line per single-grid config (32^2, 256^2, 1024^2) "
                         "and one for 1024-trap chains: plain GPU latency and the single-thread oracle")
    return ap.parse_args()


def rank_seed(seed, rank):
    """Each rank plans its own grids (weak scaling, no data-path collective)."""
    return seed + 1000 * rank


def max_over_ranks(value, device, world):
    """The slowest rank's time: the job's time."""
    if world <= 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------ oracle

def oracle_sample(insts, budget_s, threads, bird=False):
    """Plan (red-rec, or bird) + batch grids in order with the CPU oracle on
    `threads` host threads until the time budget is spent. Returns (grids
    done, seconds)."""
    import oracle
    oracle.build()

    def one(inst):
        p = (oracle.bird if bird else oracle.plan)(inst.grid, inst.rect)
        if p.status == 0:
            oracle.batch(p.moves, *inst.grid.shape)
        return 1

    t0 = time.perf_counter()
    done = 0
    it = iter(insts)
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        pending = set()
        for _ in range(threads):
            x = next(it, None)
            if x is not None:
                pending.add(ex.submit(one, x))
        while pending:
            fin, pending = cf.wait(pending, return_when=cf.FIRST_COMPLETED)
            for f in fin:
                f.result()              # re-raise oracle failures
            done += len(fin)
            if time.perf_counter() - t0 < budget_s:
                for _ in fin:
                    x = next(it, None)
                    if x is not None:
                        pending.add(ex.submit(one, x))
    return done, time.perf_counter() - t0


# ------------------------------------------------------------------ clocks

class ClockSampler:
    def __init__(self):
        self.proc = None
        self.lines = []

    def start(self, gpu_index):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


TRAFFIC_JSON = os.path.join(ROOT, "profiles", "k_sim_traffic.json")
TRAFFIC_SOURCES = ("rr_batch.cuh", "rr_batch.cu", "rr_internal.cuh")


def sources_fingerprint():
    """First 16 hex digits of sha256 over the simulation kernel's sources."""
    import hashlib
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2504_06182_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def measured_traffic_ratio(kernel):
    """DRAM bytes per algorithmic byte of `kernel` from the committed ncu
    record (profiles/k_sim_traffic.json), or None when there is none or the
    kernel's sources changed since it was taken."""
    try:
        rec = json.load(open(TRAFFIC_JSON))
        fp = sources_fingerprint()
    except Exception:
        return None
    if rec.get("kernel") != kernel or fp != rec.get("src_sha256_16"):
        return None
    return float(rec["ratio"])


def nb_alpha(ops, members):
    """Batched transfer operations of one grid's batch list (Sec. V, control
    operations): a batch in which some token takes its first elementary step
    needs one parallel extraction, a batch in which some token takes its last
    step one parallel implantation; NB_alpha counts both kinds of batches.
    ops (b, 3) = (dir, first, count), members (s,) move ids, in batch order."""
    ops = np.asarray(ops).reshape(-1, 3)
    members = np.asarray(members).reshape(-1)
    if len(members) == 0:
        return 0
    bidx = np.repeat(np.arange(len(ops)), ops[:, 2])
    _, first = np.unique(members, return_index=True)
    _, last_rev = np.unique(members[::-1], return_index=True)
    last = len(members) - 1 - last_rev
    return int(len(np.unique(bidx[first])) + len(np.unique(bidx[last])))


# ------------------------------------------------------------- paper geometry

PAPER_NTX = (32, 48, 64, 96, 128, 192, 256)
PAPER_CONTEXT = {"n_tx": 32, "cpu_us": 106, "cpu_hw": "AMD Threadripper 2950X, serial",
                 "gpu_us": 197, "gpu_hw": "Nvidia Quadro RTX 4000, one kernel"}


def paper_instances():
    """First feasible grid of seed 41 at each n_tx (n_tx columns,
    ceil(n_tx / 0.6) rows, full-width target of n_tx rows)."""
    out = []
    for n_tx in PAPER_NTX:
        for g in range(64):
            inst = gridgen.paper_instance(41, g, n_tx)
            # with a full-width target every column is a target column, so a
            # grid is feasible iff its atoms cover the target cells
            if int(inst.grid.sum()) >= n_tx * n_tx:
                out.append(inst)
                break
    return out


def median_us(fn, reps):
    t = []
    for _ in range(reps):
        t0 = time.perf_counter()
        fn()
        t.append(time.perf_counter() - t0)
    return float(np.median(t) * 1e6)


def oracle_paper_geometry():
    """Single-thread oracle latency per grid at the paper's geometry (red-rec
    plan, plan + batching, and the bird plan)."""
    import oracle
    oracle.build()
    res = {}
    for inst in paper_instances():
        reps = 20 if inst.grid.shape[1] <= 64 else 3
        plan_us = median_us(lambda: oracle.plan(inst.grid, inst.rect), reps)
        p = oracle.plan(inst.grid, inst.rect)
        both_us = median_us(lambda: oracle.batch(p.moves, *inst.grid.shape), reps) + plan_us
        bird_us = median_us(lambda: oracle.bird(inst.grid, inst.rect), reps)
        res[str(inst.grid.shape[1])] = {"plan_us": plan_us, "plan_batch_us": both_us, "bird_plan_us": bird_us}
    return res


def gpu_paper_geometry(rr, P):
    """Plain GPU latency per grid at the paper's geometry: one rr_plan call
    (grid resident on the device, counts back on the host), and rr_plan +
    rr_batch."""
    import torch
    res = {}
    for inst in paper_instances():
        m, n = inst.grid.shape
        g = torch.from_numpy(np.ascontiguousarray(gridgen.pack_bits32(inst.grid).view(np.int32))).cuda()
        cap = 2 * m * n

        def plan(bird=False):
            return P.plan(g, inst.rect, layout=rr.RR_BITS32, n=n, cap=cap, bird=bird)

        def both():
            st, mv = plan()
            if st == rr.RR_OK and len(mv):
                P.batch(mv, m, n)
            torch.cuda.synchronize()
        for _ in range(3):
            both()
            plan(True)
        reps = 50 if n <= 64 else 10
        res[str(n)] = {"plan_us": median_us(plan, reps), "plan_batch_us": median_us(both, reps),
                       "bird_plan_us": median_us(lambda: plan(True), reps)}
    return res


# ------------------------------------------------------------------ batched

def make_entries(rr, insts, grids, offs, sides, moves=None, ops=None, mem=None, caps=None):
    """Descriptors of the workload's grids (slices of one packed device
    buffer), with output slices of shared buffers when `caps` is given:
    per grid (cap moves, cap ops, cap members, move, op, member offsets)."""
    out = []
    for g, inst in enumerate(insts):
        s = sides[g]
        e = dict(grid=grids[offs[g]:offs[g + 1]], layout=rr.RR_BITS32, m=s, n=s, rect=inst.rect)
        if caps is not None:
            cm, co, cs, om, oo, os_ = caps[g]
            e.update(moves=moves[om:om + 1] if cm else None, cap_moves=cm,
                     ops=ops[oo:oo + 1] if co else None, cap_ops=co,
                     members=mem[os_:os_ + 1] if cs else None, cap_members=cs)
        out.append(e)
    return out


def sized_descriptors(rr, P, insts, grids, offs, sides, extra_flags=0):
    """Sizes every grid's outputs on the device (a planning pass without
    output room gives the move counts, a planning + batching pass with room
    for one batch per elementary step the exact step and batch counts),
    allocates them packed back to back, exactly, and returns (descriptors,
    moves, ops, members, layout); layout holds the per-grid counts and
    offsets into the packed buffers."""
    import torch
    from paper_2504_06182_gb300.planner import pack_instances, unpack_instances
    count, max_side, dev = len(insts), max(sides), grids.device
    d_inst = pack_instances(make_entries(rr, insts, grids, offs, sides))
    rr.rr_plan_batched(P.ctx, d_inst, count, max_side, extra_flags)
    torch.cuda.synchronize()
    n_moves = np.array([x.n_moves for x in unpack_instances(d_inst, count)], dtype=np.int64)
    moves = torch.empty((int(n_moves.sum()) + 1, 4), dtype=torch.int32, device=dev)
    mo = np.concatenate([[0], np.cumsum(n_moves)])
    caps = [(int(n_moves[g]), 0, 0, int(mo[g]), 0, 0) for g in range(count)]
    d_inst = pack_instances(make_entries(rr, insts, grids, offs, sides, moves, None, None, caps))
    rr.rr_plan_batched(P.ctx, d_inst, count, max_side, rr.RR_WITH_BATCH | extra_flags)
    torch.cuda.synchronize()
    n_steps = np.array([x.n_steps for x in unpack_instances(d_inst, count)], dtype=np.int64)
    so = np.concatenate([[0], np.cumsum(n_steps)])
    ops = torch.empty((int(n_steps.sum()) + 1, 3), dtype=torch.int32, device=dev)
    mem = torch.empty((int(n_steps.sum()) + 1,), dtype=torch.int32, device=dev)
    caps = [(int(n_moves[g]), int(n_steps[g]), int(n_steps[g]), int(mo[g]), int(so[g]), int(so[g]))
            for g in range(count)]
    d_inst = pack_instances(make_entries(rr, insts, grids, offs, sides, moves, ops, mem, caps))
    rr.rr_plan_batched(P.ctx, d_inst, count, max_side, rr.RR_WITH_BATCH | extra_flags)
    torch.cuda.synchronize()
    res = unpack_instances(d_inst, count)
    n_ops = np.array([x.n_ops if x.status == rr.RR_OK else 0 for x in res], dtype=np.int64)
    del ops
    oo = np.concatenate([[0], np.cumsum(n_ops)])
    ops = torch.empty((int(n_ops.sum()) + 1, 3), dtype=torch.int32, device=dev)
    caps = [(int(n_moves[g]), int(n_ops[g]), int(n_steps[g]), int(mo[g]), int(oo[g]), int(so[g]))
            for g in range(count)]
    d_inst = pack_instances(make_entries(rr, insts, grids, offs, sides, moves, ops, mem, caps))
    lay = {"n_moves": n_moves, "n_ops": n_ops, "n_steps": n_steps, "mo": mo, "oo": oo, "so": so}
    return d_inst, moves, ops, mem, lay


def nb_alpha_sample(insts, lay, ops_of, mem_of, limit=256):
    """Mean NB_alpha over the first `limit` feasible grids (ops_of(g) and
    mem_of(g) give that grid's host arrays)."""
    vals = []
    for g in range(len(insts)):
        if len(vals) >= limit:
            break
        if lay["n_steps"][g] == 0 or lay["n_ops"][g] == 0:
            continue
        vals.append(nb_alpha(ops_of(g), mem_of(g)))
    return (float(np.mean(vals)) if vals else None), len(vals)


def run_bird(args, rr, P, insts, grids, offs, sides, flush, cpu_threads):
    """The bird planner (Alg. 2) with batching on the same resident grids:
    one rr_plan_batched(RR_WITH_BATCH | RR_BIRD) call per step, L2 flushed
    between steps, CUDA events on the launching stream; its per-stage times;
    its control-operation counts next to red-rec's; the CPU oracle (bird +
    batching) on a bounded sample of the same grids."""
    import torch
    from paper_2504_06182_gb300.planner import unpack_instances
    count, max_side = len(insts), max(sides)
    flags = rr.RR_WITH_BATCH | rr.RR_BIRD
    d_inst, moves, ops, mem, lay = sized_descriptors(rr, P, insts, grids, offs, sides, rr.RR_BIRD)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        rr.rr_plan_batched(P.ctx, d_inst, count, max_side, flags, stream)
    torch.cuda.synchronize()
    rr.rr_set_tracing(P.ctx, True)
    times, stage_tot = [], {}
    with timed_region():
        for _ in range(args.steps):
            flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            st = rr.rr_plan_batched(P.ctx, d_inst, count, max_side, flags, stream)
            b.record(stream)
            b.synchronize()
            if st != rr.RR_OK:
                raise rr.RRError(st, rr.rr_last_error(P.ctx))
            times.append(a.elapsed_time(b))
            for nm, ms in rr.rr_stage_times(P.ctx):
                stage_tot[nm] = stage_tot.get(nm, 0.0) + ms
    rr.rr_set_tracing(P.ctx, False)
    res = unpack_instances(d_inst, count)
    bad = [(g, x.status) for g, x in enumerate(res) if x.status not in (rr.RR_OK, rr.RR_INFEASIBLE)]
    if bad:
        raise RuntimeError(f"bird instances failed: {bad[:5]}")
    feasible = sum(x.status == rr.RR_OK for x in res)
    tot_moves = sum(x.n_moves for x in res)
    tot_ops = sum(x.n_ops for x in res)
    tot_mem = sum(x.n_members for x in res)
    nba, nba_n = nb_alpha_sample(
        insts, lay, lambda g: ops[lay["oo"][g]:lay["oo"][g + 1]].cpu().numpy(),
        lambda g: mem[lay["so"][g]:lay["so"][g] + lay["n_steps"][g]].cpu().numpy())
    del moves, ops, mem
    cpu = None
    if not args.no_cpu_baseline:
        done, secs = oracle_sample(insts, min(args.cpu_budget, 10.0), cpu_threads, bird=True)
        cpu = {"value": done / secs, "unit": "grids/s", "cores": cpu_threads, "kind": "oracle",
               "sample": f"first {done} grids of the workload (bird + batching), {cpu_threads} host threads, "
                         f"{secs:.1f} s"}
    total_ms = float(sum(times))
    return {"value": count * args.steps / (total_ms * 1e-3), "unit": "grids/s",
            "ms_per_step": total_ms / args.steps,
            "note": "the same grids planned with bird (Alg. 2) and batched, one rr_plan_batched call per step",
            "stages_ms_per_step": {k: v / args.steps for k, v in sorted(stage_tot.items(), key=lambda kv: -kv[1])},
            "control_ops_per_feasible_grid": {
                "N_nu": tot_mem / max(1, feasible), "N_alpha": 2 * tot_moves / max(1, feasible),
                "NB_nu": tot_ops / max(1, feasible), "N_nu_per_NB_nu": tot_mem / max(1, tot_ops),
                "NB_alpha": nba, "NB_alpha_sample": f"first {nba_n} feasible grids"},
            "feasible": int(feasible), "cpu_baseline": cpu}


# ------------------------------------------------------------------ plain

def run_plain(rr, P, insts, sample):
    """One grid per call (rr_plan then rr_batch, each synchronising), the
    plain single-instance GPU path, on the first `sample` grids."""
    import torch
    from paper_2504_06182_gb300.planner import Planner  # noqa: F401
    grids = []
    for inst in insts[:sample]:
        w = gridgen.pack_bits32(inst.grid).view(np.int32)
        grids.append((torch.from_numpy(np.ascontiguousarray(w)).cuda(), inst))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for g, inst in grids:
        s_ = inst.grid.shape[0]
        st, mv = P.plan(g, inst.rect, layout=rr.RR_BITS32, n=s_, cap=2 * s_ * s_)
        if st == rr.RR_OK and len(mv):
            P.batch(mv, s_, s_)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    return {"value": len(grids) / secs, "unit": "grids/s",
            "sample": f"first {len(grids)} grids of the workload, one rr_plan + rr_batch call each"}


# ------------------------------------------------------------------ served

SERVED_SIDES = gridgen.SIDES_SERVED


def fifo_latencies(arrivals, service):
    """Latency of each request when one server takes them in arrival order:
    the plain path, one grid per call."""
    free, out = 0.0, []
    for ta, sv in zip(arrivals, service):
        start = max(ta, free)
        free = start + sv
        out.append(free - ta)
    return out


def served_grid(seed, i):
    """Request i of the served stream: (packed grid words, target rect, side)."""
    side, _ = gridgen.mixed_draw(seed, i, SERVED_SIDES, 0.6, 0.6)
    inst = gridgen.square_instance(seed, i, side, 0.6)
    return np.ascontiguousarray(gridgen.pack_bits32(inst.grid).view(np.int32)), inst.rect, side


def _served_chunk(job):
    seed, lo, hi = job
    return [served_grid(seed, i) for i in range(lo, hi)]


def served_grids(seed, n):
    """The first n requests' grids, each drawn from its own seeded stream
    (large counts on a spawned process pool: CUDA is already initialised)."""
    if n <= 2000:
        return [served_grid(seed, i) for i in range(n)]
    import multiprocessing as mp
    jobs = [(seed, lo, min(n, lo + 500)) for lo in range(0, n, 500)]
    with mp.get_context("spawn").Pool(os.cpu_count() or 4) as pool:
        parts = pool.map(_served_chunk, jobs)
    return [x for part in parts for x in part]


def run_served(rr, requests, load, seed=5, slots=256, streams=32, max_wave=8, plain_n=48, lam_n=48):
    """Served stream (C5): grids with side uniform in {64, 80, ..., 512},
    p = 0.6, centred floor(0.7 side) target, submitted from host memory;
    latency = completion - submission per request. Every request of the
    high-load run is a distinct seeded grid.

    1. plain: the first plain_n grids one at a time (H2D of the grid,
       rr_plan, rr_batch, synchronise): its maximum rate and service times;
    2. Poisson arrivals at 0.5, 0.8 and 0.95 x that rate (lam_n requests
       each, distinct grids): served p50/p99, and plain p50/p99 for the same
       arrivals from a first-in-first-out queue over the measured service
       times (cycled over the plain_n sampled grids);
    3. saturation: a burst of 192 requests at once;
    4. Poisson arrivals at `load` x the served saturation (`requests`)."""
    import torch
    from paper_2504_06182_gb300.planner import Planner
    pool = served_grids(seed, max(requests, plain_n, lam_n, 192))

    # 1. plain, one grid per call
    P = Planner(arena_bytes=2 << 30)
    service = []
    try:
        for w, rect, s_ in pool[:1] + pool[:plain_n]:          # the first call warms up
            t0 = time.perf_counter()
            g = torch.from_numpy(w).cuda()
            st, mv = P.plan(g, rect, layout=rr.RR_BITS32, n=s_, cap=2 * s_ * s_)
            if st == rr.RR_OK and len(mv):
                P.batch(mv, s_, s_)
            torch.cuda.synchronize()
            service.append(time.perf_counter() - t0)
    finally:
        P.close()
    service = service[1:]
    plain_rate = len(service) / sum(service)

    # workspace arenas: 48 GiB in total over the streams, at least 1 GiB each
    arena = max(1 << 30, (48 << 30) // streams)
    srv = rr.rr_serve_open(max_side=512, slots=slots, streams=streams, max_wave=max_wave, flags=rr.RR_WITH_BATCH,
                           arena_bytes=arena, heap_bytes=24 << 30)
    try:
        def submit(i):
            w, rect, s_ = pool[i % len(pool)]
            st, t = rr.rr_serve_submit(srv, w, rr.RR_BITS32, s_, s_, rect)
            if st != rr.RR_OK:
                raise rr.RRError(st, "rr_serve_submit")
            return t

        def drain(tickets, lat, block):
            keep = []
            for t in tickets:
                st, res = rr.rr_serve_poll(srv, t, 60_000_000 if block else 0)
                if st == rr.RR_OK:
                    if res.status not in (rr.RR_OK, rr.RR_INFEASIBLE):
                        raise rr.RRError(res.status, "served request failed")
                    lat.append(res.t_done_us - res.t_submit_us)
                    rr.rr_serve_release(srv, t)
                else:
                    keep.append(t)
            return keep

        def poisson(rate, n, index, rseed):
            arrivals = np.cumsum(np.random.default_rng(rseed).exponential(1.0 / rate, size=n))
            lat, outstanding = [], []
            t0 = time.perf_counter()
            for i, ta in enumerate(arrivals):
                # drain finished requests, then sleep until the next arrival
                # (the server's worker shares a mutex with polling: no spinning)
                while True:
                    outstanding = drain(outstanding, lat, False)
                    wait = ta - (time.perf_counter() - t0)
                    if wait <= 0:
                        break
                    time.sleep(min(wait, 0.002))
                outstanding.append(submit(index(i)))
            while outstanding:
                outstanding = drain(outstanding, lat, True)
            secs = time.perf_counter() - t0
            return arrivals, np.array(lat) / 1e3, n / secs

        # 2. arrivals at fractions of the plain rate
        vs_plain = []
        for k, frac in enumerate((0.5, 0.8, 0.95)):
            rate = frac * plain_rate
            arrivals, lat, _ = poisson(rate, lam_n, lambda i: i, seed + 10 + k)
            plat = np.array(fifo_latencies(arrivals, [service[i % plain_n] for i in range(lam_n)])) * 1e3
            vs_plain.append({"rate_per_s": rate, "fraction_of_plain_max": frac, "requests": lam_n,
                             "served_p50_ms": float(np.percentile(lat, 50)),
                             "served_p99_ms": float(np.percentile(lat, 99)),
                             "plain_p50_ms": float(np.percentile(plat, 50)),
                             "plain_p99_ms": float(np.percentile(plat, 99))})
        # 3. saturation throughput: a burst of the pool's requests at once
        nb = 192
        t0 = time.perf_counter()
        out = [submit(i) for i in range(nb)]
        drain(out, [], True)
        sat = nb / (time.perf_counter() - t0)
        # 4. Poisson arrivals at `load` x saturation
        _, lat, gps = poisson(load * sat, requests, lambda i: i, seed)
        return {"sides": "64..512 step 16", "p": 0.6,
                "server": {"slots": slots, "streams": streams, "max_wave": max_wave},
                "plain_grids_per_s": plain_rate, "plain_sample": f"first {plain_n} grids, one call each",
                "saturation_grids_per_s": sat,
                "at_fraction_of_plain": vs_plain,
                "high_load": {"rate_per_s": load * sat, "fraction_of_saturation": load, "requests": requests,
                              "grids_per_s": gps, "p50_ms": float(np.percentile(lat, 50)),
                              "p99_ms": float(np.percentile(lat, 99))},
                "note": f"{len(pool)} distinct seeded grids, request i is grid i"}
    finally:
        rr.rr_serve_close(srv)


# ------------------------------------------------------------------ ours

def run_ours(args, rank, world, local):
    import torch
    import paper_2504_06182_gb300 as rr
    from paper_2504_06182_gb300.planner import Planner, unpack_instances

    insts = gridgen.mixed_instances(rank_seed(args.seed, rank), args.count)
    # CPU oracle baseline on host cores before any GPU work (rank 0, N = 1)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        done, secs = oracle_sample(insts, args.cpu_budget, threads)
        cpu = {"value": done / secs, "unit": "grids/s", "cores": threads, "kind": "oracle",
               "sample": f"first {done} grids of the workload (plan + batching), {threads} host threads, "
                         f"{secs:.1f} s",
               "paper_geometry_1thread": oracle_paper_geometry()}

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl", device_id=dev)

    # packed grids: one pinned host buffer, one device buffer
    words = [gridgen.pack_bits32(i.grid).view(np.int32).ravel() for i in insts]
    offs = np.cumsum([0] + [len(w) for w in words])
    host = torch.empty(int(offs[-1]), dtype=torch.int32).pin_memory()
    host.numpy()[:] = np.concatenate(words)
    grids = host.to(dev)
    count = len(insts)
    sides = [i.grid.shape[0] for i in insts]
    max_side = max(sides)

    P = Planner(arena_bytes=int(os.environ.get("RR_ARENA_GB", "24")) << 30)
    d_inst, moves, ops, mem, lay = sized_descriptors(rr, P, insts, grids, offs, sides)
    inst_host = d_inst.cpu().pin_memory()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2

    stream = torch.cuda.current_stream()

    def step():
        st = rr.rr_plan_batched(P.ctx, d_inst, count, max_side, rr.RR_WITH_BATCH, stream)
        if st != rr.RR_OK:
            raise rr.RRError(st, rr.rr_last_error(P.ctx))

    # launch configuration picked by the library's autotuner on this workload
    # (before the warm-up; not timed)
    tuned_nclass, tuned_shift, tuned_pipe = (4, 0, 1) if args.no_autotune else \
        rr.rr_autotune(P.ctx, d_inst, count, max_side, rr.RR_WITH_BATCH, stream)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    res = unpack_instances(d_inst, count)
    bad = [(g, x.status) for g, x in enumerate(res) if x.status not in (rr.RR_OK, rr.RR_INFEASIBLE)]
    if bad:
        raise RuntimeError(f"instances failed: {bad[:5]}")

    rr.rr_set_tracing(P.ctx, True)
    launches0 = rr.rr_launch_count(P.ctx)
    stage_tot = {}
    times = []
    clocks = ClockSampler()
    if rank == 0:
        clocks.start(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with timed_region():
        for _ in range(args.steps):
            flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step()
            b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b))
            for nm, ms in rr.rr_stage_times(P.ctx):
                stage_tot[nm] = stage_tot.get(nm, 0.0) + ms
    torch.cuda.synchronize()
    launches = rr.rr_launch_count(P.ctx) - launches0
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop() if rank == 0 else None
    rr.rr_set_tracing(P.ctx, False)
    elapsed_ms = max_over_ranks(sum(times), dev, world)

    # the same step replayed from a captured CUDA graph (RR_GRAPH), under the
    # configuration the autotuner picks for replays
    gflags = rr.RR_WITH_BATCH | rr.RR_GRAPH
    graph_cfg = None if args.no_autotune else rr.rr_autotune(P.ctx, d_inst, count, max_side, gflags, stream)
    if rr.rr_plan_batched(P.ctx, d_inst, count, max_side, gflags, stream) != rr.RR_OK:
        raise rr.RRError(-3, rr.rr_last_error(P.ctx))
    torch.cuda.synchronize()
    graph_ms = []
    with timed_region():
        for _ in range(args.steps):
            flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            rr.rr_plan_batched(P.ctx, d_inst, count, max_side, gflags, stream)
            b.record(stream)
            b.synchronize()
            graph_ms.append(a.elapsed_time(b))
    graph_total = float(sum(graph_ms))

    res = unpack_instances(d_inst, count)
    tot_moves = sum(x.n_moves for x in res)
    tot_ops = sum(x.n_ops for x in res)
    tot_mem = sum(x.n_members for x in res)
    feasible = sum(x.status == rr.RR_OK for x in res)

    # end to end through the public call with host buffers: every step copies
    # the packed grids and descriptors in from pinned host memory, makes the
    # call, and copies every move, batch and member and the descriptors
    # (statuses, counts) back to pinned host memory. The copies back run on a
    # copy stream; consecutive steps alternate between two sets of device
    # output buffers (and of host buffers), so that one step's copy back
    # overlaps the next step's call. The timed region runs from the first
    # step's copy in to the end of the last step's copy back.
    from paper_2504_06182_gb300.planner import pack_instances
    nm_, no_, ns_ = int(lay["n_moves"].sum()), int(lay["n_ops"].sum()), int(lay["n_steps"].sum())
    caps = [(int(lay["n_moves"][g]), int(lay["n_ops"][g]), int(lay["n_steps"][g]), int(lay["mo"][g]),
             int(lay["oo"][g]), int(lay["so"][g])) for g in range(count)]
    copy_stream = torch.cuda.Stream(device=dev)
    bufs = []
    for bi in range(2):
        mv_d, op_d, me_d = (moves, ops, mem) if bi == 0 else \
            (torch.empty_like(moves), torch.empty_like(ops), torch.empty_like(mem))
        di = pack_instances(make_entries(rr, insts, grids, offs, sides, mv_d, op_d, me_d, caps))
        bufs.append({"moves": mv_d, "ops": op_d, "mem": me_d, "inst": di, "inst_h": di.cpu().pin_memory(),
                     "back": torch.empty((di.numel(),), dtype=torch.uint8, pin_memory=True),
                     "moves_h": torch.empty((nm_, 4), dtype=torch.int32, pin_memory=True),
                     "ops_h": torch.empty((no_, 3), dtype=torch.int32, pin_memory=True),
                     "mem_h": torch.empty((ns_,), dtype=torch.int32, pin_memory=True),
                     "done": torch.cuda.Event()})
    h2d = host.numel() * 4 + bufs[0]["inst_h"].numel()
    d2h = bufs[0]["inst_h"].numel() + 4 * (4 * nm_ + 3 * no_ + ns_)

    issued = []

    def e2e_step(i):
        B = bufs[i % 2]
        # the host stays at most one step ahead: it issues step i once step
        # i - 2's call has finished (queues stay shallow; step i - 1 keeps the
        # GPU busy meanwhile)
        if len(issued) >= 2:
            issued[-2].synchronize()
        stream.wait_event(B["done"])            # that buffer set's previous copy back has finished
        grids.copy_(host, non_blocking=True)
        B["inst"].copy_(B["inst_h"], non_blocking=True)
        st = rr.rr_plan_batched(P.ctx, B["inst"], count, max_side, rr.RR_WITH_BATCH, stream)
        if st != rr.RR_OK:
            raise rr.RRError(st, rr.rr_last_error(P.ctx))
        called = torch.cuda.Event()
        called.record(stream)
        issued.append(called)
        del issued[:-2]
        copy_stream.wait_event(called)
        with torch.cuda.stream(copy_stream):
            B["back"].copy_(B["inst"], non_blocking=True)
            B["moves_h"].copy_(B["moves"][:nm_], non_blocking=True)
            B["ops_h"].copy_(B["ops"][:no_], non_blocking=True)
            B["mem_h"].copy_(B["mem"][:ns_], non_blocking=True)
        B["done"].record(copy_stream)

    # the direct launches of this leg use the configuration tuned for direct
    # launches (the graph leg left the one tuned for replays)
    if not args.no_autotune:
        rr.rr_set_config(P.ctx, tuned_nclass, tuned_shift, tuned_pipe)
    # warm-up: the timed loop's own body (the host pages are touched, every
    # first use in the process happens here), twice over both buffer sets
    for i in range(max(4, args.warmup)):
        flush.fill_(1)
        e2e_step(i)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    with timed_region():
        a.record(stream)
        for i in range(args.steps):
            flush.fill_(1)
            e2e_step(i)
        b.record(copy_stream)
        b.synchronize()
    torch.cuda.synchronize()
    e2e_total = max_over_ranks(a.elapsed_time(b), dev, world)
    last = bufs[(args.steps - 1) % 2]
    from paper_2504_06182_gb300 import rr_instance
    res_e2e = (rr_instance * count).from_buffer_copy(last["back"].numpy().tobytes())
    bad = [(g, x.status) for g, x in enumerate(res_e2e) if x.status not in (rr.RR_OK, rr.RR_INFEASIBLE)]
    if bad:
        raise RuntimeError(f"end-to-end instances failed: {bad[:5]}")
    ops_np, mem_np = last["ops_h"].numpy(), last["mem_h"].numpy()
    nba, nba_n = nb_alpha_sample(insts, lay, lambda g: ops_np[lay["oo"][g]:lay["oo"][g + 1]],
                                 lambda g: mem_np[lay["so"][g]:lay["so"][g] + lay["n_steps"][g]])
    del ops_np, mem_np, last, bufs

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    plain = run_plain(rr, P, insts, args.plain_sample) if args.plain_sample > 0 else None
    paper = {"gpu": gpu_paper_geometry(rr, P), "paper_context": PAPER_CONTEXT,
             "geometry": "n_tx columns, ceil(n_tx/0.6) rows, full-width target of n_tx rows, p = 0.6"} \
        if args.plain_sample > 0 else None
    del ops, mem, moves
    bird = run_bird(args, rr, P, insts, grids, offs, sides, flush, os.cpu_count() or 1) \
        if not args.no_bird else None
    P.close()
    torch.cuda.empty_cache()
    served = run_served(rr, args.served_requests, args.served_load, plain_n=min(48, args.served_plain_requests),
                        lam_n=args.served_plain_requests) if args.served_requests > 0 else None

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak_gbs = float(peaks.get("hbm_gbs", 6800.0))
    # dominant kernel and its algorithmic bytes per launch
    dom = max(stage_tot, key=stage_tot.get) if stage_tot else None
    grid_bytes = host.numel() * 4
    alg = {
        "k_sim": 16 * tot_moves + 12 * tot_ops + 4 * tot_mem,
        "k_emit_recv": 16 * tot_moves,
        "k_transpose": 2 * grid_bytes,
    }
    roof = None
    if dom is not None:
        avg_ms = stage_tot[dom] / args.steps
        byt = alg.get(dom)
        if byt is not None:
            ach = byt / (avg_ms * 1e-3) / 1e9
            ratio = measured_traffic_ratio(dom)
            roof = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": peak_gbs, "unit": "GB/s",
                    "frac": ach / peak_gbs, "traffic": int(ratio * byt) if ratio else None,
                    "peak_source": "measured" if peaks else "fallback",
                    "alg_bytes_per_launch": int(byt), "avg_ms": avg_ms,
                    "launch": "one step's simulation: every simulation launch of the step (pipeline groups "
                              "and size classes), timed from the first one's start to the join after the last"
                              if dom == "k_sim" else "one launch"}
    value = count * world * args.steps / (elapsed_ms * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": "grids/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grids_per_gpu": count, "layout": "bits32", "seed": args.seed,
                   "l2": "flushed between steps (256 MiB write)", "parallelism": f"dp{world}",
                   "autotuned": None if args.no_autotune else {"size_classes": tuned_nclass,
                                                               "block_budget_scale": 2.0 ** tuned_shift,
                                 "largest_first": ["off", "1/4", "1/16, 1/4", "1/16, 1/8, 1/4, 1/2", "1/64, 1/16, 1/4"][tuned_pipe]}},
        "e2e": {"value": count * world * args.steps / (e2e_total * 1e-3), "unit": "grids/s",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "note": "per step: H2D of the packed grids and descriptors from pinned host memory, the call, "
                        "D2H of every move, batch and member and the descriptors to pinned host memory on a copy "
                        "stream; steps alternate between two output buffer sets so that one step's D2H overlaps "
                        "the next step's call; timed from the first H2D to the end of the last D2H"},
        "gpu_launches": launches,
        "graph": {"value": count * args.steps / (graph_total * 1e-3), "unit": "grids/s",
                  "autotuned_for_replay": None if graph_cfg is None else
                  {"size_classes": graph_cfg[0], "block_budget_scale": 2.0 ** graph_cfg[1], "split": graph_cfg[2]},
                  "note": "same step replayed from one captured CUDA graph (RR_GRAPH), inputs resident"},
        "roofline": roof,
        "cpu_baseline": cpu,
        "plain": plain,
        "paper_geometry": paper,
        "served": served,
        "bird": bird,
        "clocks": clk,
        "stages_ms_per_step": {k: v / args.steps for k, v in sorted(stage_tot.items(), key=lambda kv: -kv[1])},
        "totals_per_step": {"moves": int(tot_moves), "ops": int(tot_ops), "steps": int(tot_mem),
                            "feasible": int(feasible), "grids": count},
        # control operations of one reconfiguration cycle (§V): displacement
        # operations N_nu = elementary steps, transfer operations N_alpha = one
        # extraction and one implantation per move, batched displacement
        # sequences NB_nu = batches, batched transfers NB_alpha = batches with
        # a first step (one parallel extraction) plus batches with a last step
        # (one parallel implantation), on a sample of the grids
        "control_ops_per_feasible_grid": {
            "N_nu": tot_mem / max(1, feasible), "N_alpha": 2 * tot_moves / max(1, feasible),
            "NB_nu": tot_ops / max(1, feasible), "N_nu_per_NB_nu": tot_mem / max(1, tot_ops),
            "NB_alpha": nba, "NB_alpha_sample": f"first {nba_n} feasible grids"},
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# ------------------------------------------------------------------ reference

def run_reference(args, rank, world):
    if rank != 0:
        return
    insts = gridgen.mixed_instances(args.seed, args.count)
    threads = os.cpu_count() or 1
    budget = float(os.environ.get("RR_REF_STEP_S", "8"))
    for _ in range(args.warmup):
        oracle_sample(insts[:threads], budget / 4, threads)
    done_tot, secs_tot = 0, 0.0
    for s in range(args.steps):
        # each step a bounded sample: consecutive grids from a rotating start
        start = (s * 97) % max(1, len(insts) - 1)
        done, secs = oracle_sample(insts[start:] + insts[:start], budget, threads)
        done_tot += done
        secs_tot += secs
    value = done_tot / secs_tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "grids/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs_tot * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grids_per_gpu": args.count, "layout": "bits32", "seed": args.seed},
        "cpu_baseline": {"value": value, "unit": "grids/s", "cores": threads, "kind": "oracle",
                         "sample": f"{done_tot} grids over {args.steps} steps of ~{budget:.0f} s, "
                                   f"{threads} host threads"},
        "e2e": {"value": value, "unit": "grids/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------- single-grid configs

SINGLE_CONFIGS = (
    ("32x32 u8, p = 0.6, centred 20x20 target", 32, 20, "u8"),
    ("256x256 u8, p = 0.6, centred 180x180 target", 256, 180, "u8"),
    ("1024x1024 bits32, p = 0.6, centred 720x720 target", 1024, 720, "bits32"),
)


def path_steps(moves):
    return int((np.abs(moves[:, 0] - moves[:, 2]) + np.abs(moves[:, 1] - moves[:, 3])).sum()) if len(moves) else 0


def run_configs(args):
    """Plain per-grid latency of each single-grid config on seeds 0..9 (GPU:
    one rr_plan call, and rr_plan + rr_batch, grid resident on the device)
    and, as this mode's CPU baseline, the single-thread oracle on the same
    grids (1024^2: planning on seeds 0..2 and the first 200 000 batches of
    seed 0, a bounded sample). Medians over seeds."""
    import oracle
    oracle.build()
    seeds = list(range(10))
    cpu = {}
    for name, side, t, _ in SINGLE_CONFIGS:
        plan_us, both_us, bird_us, sample = [], [], [], ""
        for sd in (seeds if side < 1024 else seeds[:3]):
            inst = gridgen.square_instance(sd, 0, side, 0.6, t)
            t0 = time.perf_counter()
            p = oracle.plan(inst.grid, inst.rect)
            t1 = time.perf_counter()
            plan_us.append((t1 - t0) * 1e6)
            if side < 1024:
                oracle.batch(p.moves, side, side, cap=path_steps(p.moves))
                both_us.append((time.perf_counter() - t0) * 1e6)
                # the oracle's bird scans every window: too slow beyond 256^2
                tb = time.perf_counter()
                oracle.bird(inst.grid, inst.rect)
                bird_us.append((time.perf_counter() - tb) * 1e6)
            elif sd == 0:
                t2 = time.perf_counter()
                ops, _ = oracle.batch(p.moves, side, side, max_ops=200000, cap=path_steps(p.moves))
                rate = len(ops) / (time.perf_counter() - t2)
                sample = f"planning on seeds 0..2; batching: the first {len(ops)} batches of seed 0 " \
                         f"at {rate:.0f} batches/s"
        cpu[side] = {"kind": "oracle", "cores": 1, "plan_us": float(np.median(plan_us)),
                     "plan_batch_us": float(np.median(both_us)) if both_us else None,
                     "bird_plan_us": float(np.median(bird_us)) if bird_us else None,
                     "sample": sample or f"seeds 0..{seeds[-1]}, one grid at a time"}
    cpu_chain = oracle_chain_us()
    import torch
    import paper_2504_06182_gb300 as rr
    from paper_2504_06182_gb300.planner import Planner
    P = Planner(arena_bytes=4 << 30)
    for name, side, t, lay in SINGLE_CONFIGS:
        layout = rr.RR_U8 if lay == "u8" else rr.RR_BITS32
        plan_us, both_us, bird_us, outs = [], [], [], None
        one_plan_us, one_both_us = [], []
        for sd in seeds:
            inst = gridgen.square_instance(sd, 0, side, 0.6, t)
            host = inst.grid if lay == "u8" else gridgen.pack_bits32(inst.grid).view(np.int32)
            g = torch.from_numpy(np.ascontiguousarray(host)).cuda()
            cap = 2 * side * side
            if side <= rr.RR_ONE_MAX_SIDE:
                # the one-launch path, outputs sized beforehand (a real-time
                # loop keeps its buffers): plan, and plan + batching
                st, mv = P.plan(g, inst.rect, layout=layout, n=side, cap=cap)
                k = max(1, len(mv))
                nst = max(1, path_steps(mv.cpu().numpy())) if len(mv) else 1
                o_mv = torch.empty((k, 4), dtype=torch.int32, device="cuda")
                o_ops = torch.empty((nst, 3), dtype=torch.int32, device="cuda")
                o_mem = torch.empty((nst,), dtype=torch.int32, device="cuda")

                def one(flags):
                    r = rr.rr_plan_one(P.ctx, g, layout, side, side, inst.rect, flags, o_mv, k, o_ops, nst, o_mem, nst)
                    if r[0] not in (rr.RR_OK, rr.RR_INFEASIBLE):
                        raise rr.RRError(r[0], rr.rr_last_error(P.ctx))
                    return r
                one(rr.RR_WITH_BATCH)
                one_plan_us.append(median_us(lambda: one(0), 20))
                one_both_us.append(median_us(lambda: one(rr.RR_WITH_BATCH), 20 if side <= 64 else 3))

            def plan():
                r = P.plan(g, inst.rect, layout=layout, n=side, cap=cap)
                torch.cuda.synchronize()
                return r

            def both():
                st, mv = plan()
                res = P.batch(mv, side, side) if st == rr.RR_OK and len(mv) else None
                torch.cuda.synchronize()
                return st, mv, res
            def bird():
                r = P.plan(g, inst.rect, layout=layout, n=side, cap=cap, bird=True)
                torch.cuda.synchronize()
                return r
            both()
            bird()
            reps = 20 if side <= 256 else 2
            plan_us.append(median_us(plan, reps))
            both_us.append(median_us(both, max(2, reps // 4)))
            bird_us.append(median_us(bird, reps))
            if sd == 0:
                st, mv, res = both()
                outs = {"status": int(st), "moves": int(len(mv)),
                        "ops": int(len(res[0])) if res else 0, "steps": int(len(res[1])) if res else 0}
        line = {"config": name, "metric": "plain per-grid latency (median over seeds 0..9)", "unit": "us",
                "gpu": {"plan_us": float(np.median(plan_us)), "plan_batch_us": float(np.median(both_us)),
                        "bird_plan_us": float(np.median(bird_us)),
                        "path": "one rr_plan (and rr_batch) call per grid, grid resident on the device, synchronised"},
                "gpu_one_launch": {"plan_us": float(np.median(one_plan_us)),
                                   "plan_batch_us": float(np.median(one_both_us)),
                                   "path": "one rr_plan_one call (a single kernel launch) per grid, outputs "
                                           "allocated beforehand, synchronised"} if one_plan_us else None,
                "cpu_baseline": cpu[side], "seed0_outputs": outs, "data": "synthetic"}
        print(json.dumps(line), flush=True)
    run_chains(rr, P, cpu_chain)
    P.close()


CHAIN_TRAPS = 1024
CHAIN_COUNT = 16384


def oracle_chain_us():
    """Single-thread oracle latency of one 1024-trap chain (median of 200)."""
    import oracle
    inst = gridgen.chain_instance(0, 0, CHAIN_TRAPS)
    return median_us(lambda: oracle.plan(inst.grid, inst.rect), 200)


def run_chains(rr, P, cpu_us):
    """The paper's 1D workload: chains of 1024 traps with a centred target of
    512 (eta = 0.5), fill 0.6. One chain per rr_plan call, and 16384 chains
    per rr_plan_batched call (planning only: the exact 1D solve)."""
    import torch
    from paper_2504_06182_gb300.planner import pack_instances, unpack_instances
    one = gridgen.chain_instance(0, 0, CHAIN_TRAPS)
    g1 = torch.from_numpy(np.ascontiguousarray(one.grid)).cuda()

    def plan1():
        r = P.plan(g1, one.rect, layout=rr.RR_U8, n=1, cap=2 * CHAIN_TRAPS)
        torch.cuda.synchronize()
        return r
    plan1()
    plain_us = median_us(plan1, 200)
    insts = [gridgen.chain_instance(1, g, CHAIN_TRAPS) for g in range(CHAIN_COUNT)]
    grids = torch.from_numpy(np.ascontiguousarray(np.concatenate([i.grid.ravel() for i in insts]))).cuda()
    moves = torch.empty((CHAIN_COUNT * 2 * CHAIN_TRAPS, 4), dtype=torch.int32, device="cuda")
    entries = [dict(grid=grids[g * CHAIN_TRAPS:(g + 1) * CHAIN_TRAPS], layout=rr.RR_U8, m=CHAIN_TRAPS, n=1,
                    rect=insts[g].rect, moves=moves[g * 2 * CHAIN_TRAPS:], cap_moves=2 * CHAIN_TRAPS)
               for g in range(CHAIN_COUNT)]
    dev = pack_instances(entries)
    stream = torch.cuda.current_stream()
    times = []
    for it in range(6):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        rr.rr_plan_batched(P.ctx, dev, CHAIN_COUNT, CHAIN_TRAPS, 0, stream)
        b.record(stream)
        b.synchronize()
        if it:
            times.append(a.elapsed_time(b))
    res = unpack_instances(dev, CHAIN_COUNT)
    bad = sum(x.status not in (rr.RR_OK, rr.RR_INFEASIBLE) for x in res)
    line = {"config": f"chains of {CHAIN_TRAPS} traps, centred target of {CHAIN_TRAPS // 2} (eta 0.5), p = 0.6",
            "metric": "exact 1D solve: per-chain latency and batched chains/s", "unit": "us, chains/s",
            "gpu": {"plan_us": plain_us,
                    "batched_chains_per_s": CHAIN_COUNT / (float(np.median(times)) * 1e-3),
                    "batched": f"{CHAIN_COUNT} chains per rr_plan_batched call, median of 5", "failed": int(bad)},
            "cpu_baseline": {"kind": "oracle", "cores": 1, "plan_us": cpu_us, "sample": "one chain, median of 200"},
            "paper_context": {"cpu_serial_us": 22, "hw": "AMD Threadripper 2950X"},
            "data": "synthetic (Bernoulli loading stands in for the paper's exact 0.6 n_t atoms)"}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.configs:
        if rank == 0:
            run_configs(args)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
