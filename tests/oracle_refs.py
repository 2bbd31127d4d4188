"""Expected outputs from the oracle for many grids at once (test helper).

The oracle is plain sequential C called through ctypes, which releases the
GIL, so independent grids are planned and batched on a thread pool (threads,
not forked processes: the GPU tests have CUDA initialised by then)."""
from __future__ import annotations

import concurrent.futures as cf
import os
from dataclasses import dataclass

import numpy as np

import oracle


@dataclass
class Ref:
    status: int
    moves: np.ndarray
    ops: np.ndarray | None
    members: np.ndarray | None


def _one(grid, rect, bird, strict, with_batch):
    p = (oracle.bird if bird else oracle.plan)(grid, rect, strict=strict)
    ops = mem = None
    if with_batch and p.status == 0:
        ops, mem = oracle.batch(p.moves, *grid.shape)
    return Ref(p.status, p.moves, ops, mem)


def refs(cases, bird=False, strict=False, with_batch=True, threads=None):
    """cases: iterable of (grid, rect). Returns one Ref per case, in order."""
    oracle.lib()                       # build / load once, before the threads
    threads = threads or min(32, os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        futs = [ex.submit(_one, g, r, bird, strict, with_batch) for g, r in cases]
        return [f.result() for f in futs]


def path_steps(moves) -> int:
    mv = np.asarray(moves, dtype=np.int64).reshape(-1, 4)
    return int((np.abs(mv[:, 0] - mv[:, 2]) + np.abs(mv[:, 1] - mv[:, 3])).sum())
