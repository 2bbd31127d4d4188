"""Pins of the oracle's batching routine (Alg. 4 with the local constraints of
Sec. IV), CPU only.

P7 batches <= elementary steps (Alg. 4 deletes at least one edge per
iteration); P8 conservation (every elementary step appears in exactly one
batch) and replay equivalence; P9 the per-batch constraints; and the oracle's
dependency bookkeeping against Gamma taken literally (every earlier path that
shares a vertex), on tiny inputs.
"""
import numpy as np
import pytest

import gridgen
import oracle
from tests.checks import batch_bruteforce, replay_moves, replay_ops, path_len

RNG = np.random.default_rng(7)


def small_plans(count, mmax=9, nmax=9):
    out = []
    while len(out) < count:
        m, n = int(RNG.integers(2, mmax + 1)), int(RNG.integers(2, nmax + 1))
        grid = (RNG.random((m, n)) < RNG.uniform(0.4, 0.85)).astype(np.uint8)
        h = int(RNG.integers(1, m))
        r0 = int(RNG.integers(0, m - h + 1))
        w = int(RNG.integers(1, n + 1))
        c0 = int(RNG.integers(0, n - w + 1))
        rect = (r0, c0, r0 + h, c0 + w)
        res = oracle.plan(grid, rect)
        if res.status == 0 and 0 < len(res.moves) <= 60:
            out.append((grid, rect, res.moves))
    return out


def test_batching_matches_literal_gamma():
    for grid, rect, moves in small_plans(250):
        ops, mem = oracle.batch(moves, *grid.shape)
        bops, bmem = batch_bruteforce(moves)
        assert ops.tolist() == bops.tolist()
        assert mem.tolist() == bmem.tolist()


def test_batching_random_move_lists():
    """Alg. 4 is defined for any valid ordered path system, not only red-rec
    output: random unobstructed move sequences on random grids."""
    for trial in range(150):
        m, n = int(RNG.integers(2, 8)), int(RNG.integers(2, 8))
        g = (RNG.random((m, n)) < 0.5).astype(np.uint8)
        moves = []
        for _ in range(40):
            occ = np.argwhere(g == 1)
            free = np.argwhere(g == 0)
            if not len(occ) or not len(free):
                break
            sr, sc = occ[RNG.integers(len(occ))]
            dr, dc = free[RNG.integers(len(free))]
            mv = (int(sr), int(sc), int(dr), int(dc))
            try:
                g = replay_moves(g, None, [mv])
            except AssertionError:
                continue
            moves.append(mv)
        if not moves:
            continue
        moves = np.array(moves, dtype=np.int32)
        ops, mem = oracle.batch(moves, m, n)
        bops, bmem = batch_bruteforce(moves)
        assert ops.tolist() == bops.tolist() and mem.tolist() == bmem.tolist()


@pytest.mark.parametrize("side,target,seeds", [(32, 20, range(4)), (64, 44, range(2)), (128, 89, range(1))])
def test_batching_replay_and_conservation(side, target, seeds):
    for seed in seeds:
        inst = gridgen.square_instance(seed, 0, side, 0.6, target)
        res = oracle.plan(inst.grid, inst.rect)
        assert res.status == 0
        ops, mem = oracle.batch(res.moves, side, side)
        steps = path_len(res.moves)
        assert int(ops[:, 2].sum()) == steps == len(mem)            # P8 conservation
        assert len(ops) <= steps                                     # P7
        assert (ops[:, 1] == np.concatenate([[0], np.cumsum(ops[:, 2])[:-1]])).all()
        final_moves = replay_moves(inst.grid, inst.rect, res.moves)
        final_ops = replay_ops(inst.grid, res.moves, ops, mem)       # P9 inside
        assert (final_moves == final_ops).all()                      # P8 replay


def test_batching_leader_is_lowest_unfinished():
    """Consequence of Gamma: the lowest-id unfinished path is always ready,
    so every batch's first member is the lowest-id path not yet completed."""
    inst = gridgen.square_instance(5, 0, 48, 0.6, 33)
    res = oracle.plan(inst.grid, inst.rect)
    ops, mem = oracle.batch(res.moves, 48, 48)
    L = np.abs(res.moves[:, 0] - res.moves[:, 2]) + np.abs(res.moves[:, 1] - res.moves[:, 3])
    left = L.copy()
    lowest = 0
    for (d, f, c) in ops:
        while left[lowest] == 0:
            lowest += 1
        assert mem[f] == lowest
        left[mem[f:f + c]] -= 1


def test_batch_rejects_bad_moves():
    with pytest.raises(RuntimeError):
        oracle.batch(np.array([[0, 0, 0, 0]], dtype=np.int32), 2, 2)      # isolated
    with pytest.raises(RuntimeError):
        oracle.batch(np.array([[0, 0, 5, 0]], dtype=np.int32), 2, 2)      # off grid
    ops, mem = oracle.batch(np.zeros((0, 4), dtype=np.int32), 3, 3)
    assert len(ops) == 0 and len(mem) == 0
