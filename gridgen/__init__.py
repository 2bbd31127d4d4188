"""Seeded synthetic occupancy grids shared by the tests, the benchmark and the
smoke check.

This module holds no part of the planning method. It only draws the inputs:
0/1 trap-occupancy grids loaded i.i.d. Bernoulli(p), as in the paper's
benchmarks (Sec. V.A: random initial configurations at loading efficiency
0.6), and the centred target rectangles the workloads use.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used counter-style: the k-th
output of the stream seeded with ``state`` is ``mix64(state + (k + 1) * GAMMA)``.
Grid ``g`` of a run with seed ``seed`` uses ``state = seed ^ (g * GAMMA)``;
trap ``(r, c)`` of an ``m x n`` grid is occupied iff
``(output[r * n + c] >> 32) < thr`` with the integer threshold
``thr = floor(p * 2**32)``. Per-grid draws (side, p) of mixed-size workloads
use outputs ``2**32 + k``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
MASK64 = (1 << 64) - 1
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB


def mix64(z):
    """SplitMix64 output function on uint64 numpy arrays (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_M2)
        z = z ^ (z >> np.uint64(31))
    return z


def stream_state(seed: int, g: int) -> int:
    return (seed ^ (g * GAMMA)) & MASK64


def outputs(state: int, k) -> np.ndarray:
    """k-th outputs (array of indices) of the SplitMix64 stream seeded with state."""
    k = np.asarray(k, dtype=np.uint64)
    with np.errstate(over="ignore"):
        x = np.uint64(state) + (k + np.uint64(1)) * np.uint64(GAMMA)
    return mix64(x)


def threshold(p: float) -> int:
    """Integer occupancy threshold floor(p * 2**32), clamped to [0, 2**32]."""
    return max(0, min(1 << 32, int(math.floor(p * 4294967296.0))))


def grid_u8(seed: int, g: int, m: int, n: int, thr: int) -> np.ndarray:
    """m x n uint8 grid (row-major), 1 = trap holds an atom."""
    idx = np.arange(m * n, dtype=np.uint64)
    hi = outputs(stream_state(seed, g), idx) >> np.uint64(32)
    return (hi < np.uint64(thr)).astype(np.uint8).reshape(m, n)


def pack_bits32(grid: np.ndarray) -> np.ndarray:
    """Bit-pack a 0/1 (m, n) grid into uint32 rows: bit c & 31 of word c >> 5,
    least significant bit first, row stride ceil(n / 32) words."""
    grid = np.asarray(grid, dtype=np.uint8)
    m, n = grid.shape
    wpr = (n + 31) // 32
    pad = np.zeros((m, wpr * 32), dtype=np.uint8)
    pad[:, :n] = grid
    bits = np.packbits(pad.reshape(m, wpr, 4, 8), axis=3, bitorder="little")
    return bits.reshape(m, wpr, 4).copy().view("<u4").reshape(m, wpr)


def unpack_bits32(words: np.ndarray, n: int) -> np.ndarray:
    words = np.ascontiguousarray(words, dtype="<u4")
    m, wpr = words.shape
    b = np.unpackbits(words.view(np.uint8).reshape(m, wpr * 4), axis=1, bitorder="little")
    return b[:, :n].astype(np.uint8)


def centred_rect(m: int, n: int, h: int, w: int):
    """Half-open target rectangle (r0, c0, r1, c1) of h rows and w columns,
    centred: r0 = floor((m - h) / 2), c0 = floor((n - w) / 2)."""
    r0 = (m - h) // 2
    c0 = (n - w) // 2
    return (r0, c0, r0 + h, c0 + w)


@dataclass(frozen=True)
class Instance:
    grid: np.ndarray          # (m, n) uint8
    rect: tuple               # (r0, c0, r1, c1)
    seed: int
    g: int
    p: float


def square_instance(seed: int, g: int, side: int, p: float, target: int | None = None) -> Instance:
    """Square grid of the given side, fill p, centred square target of side
    `target` (default floor(0.7 * side))."""
    t = int(math.floor(0.7 * side)) if target is None else target
    grid = grid_u8(seed, g, side, side, threshold(p))
    return Instance(grid, centred_rect(side, side, t, t), seed, g, p)


def paper_instance(seed: int, g: int, n_tx: int, p: float = 0.6) -> Instance:
    """The paper's runtime geometry: n_tx columns and ceil(n_tx / 0.6) rows
    (integer form: (5 n_tx + 2) // 3), fill p, a full-width target of n_tx
    rows centred vertically."""
    m = (5 * n_tx + 2) // 3
    grid = grid_u8(seed, g, m, n_tx, threshold(p))
    return Instance(grid, centred_rect(m, n_tx, n_tx, n_tx), seed, g, p)


def chain_instance(seed: int, g: int, n_t: int, p: float = 0.6) -> Instance:
    """The paper's 1D workload: a chain of n_t traps (an n_t x 1 grid), fill p,
    a centred target of n_t / 2 traps (eta = 0.5). The paper loads exactly
    0.6 n_t atoms at random; Bernoulli(p) loading stands in for that."""
    grid = grid_u8(seed, g, n_t, 1, threshold(p))
    return Instance(grid, centred_rect(n_t, 1, n_t // 2, 1), seed, g, p)


def mixed_draw(seed: int, g: int, sides, p_lo: float, p_hi: float):
    """Per-grid (side, p) for mixed-size workloads: side uniform over `sides`,
    p uniform in [p_lo, p_hi], both from outputs 2**32 and 2**32 + 1 of grid
    g's stream."""
    st = stream_state(seed, g)
    u = outputs(st, np.array([1 << 32, (1 << 32) + 1], dtype=np.uint64))
    side = int(sides[int(u[0] % np.uint64(len(sides)))])
    frac = float(int(u[1] >> np.uint64(11))) * (1.0 / 9007199254740992.0)
    return side, p_lo + (p_hi - p_lo) * frac


# Workloads, named by what they are (sizes as in the benchmark definitions).
SIDES_MIXED = tuple(range(32, 257, 16))      # 32, 48, ..., 256
SIDES_SERVED = tuple(range(64, 513, 16))     # 64, 80, ..., 512


def mixed_instances(seed: int, count: int, sides=SIDES_MIXED, p_lo=0.5, p_hi=0.7):
    out = []
    for g in range(count):
        side, p = mixed_draw(seed, g, sides, p_lo, p_hi)
        out.append(square_instance(seed, g, side, p))
    return out
