"""ctypes wrapper of the sequential CPU oracle (rr_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baselines (its cpu_baseline legs and its reference arm) are the only users of
this package. The CUDA library and its Python binding never import it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rr_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

OK, INFEASIBLE, ERR_ARG, ERR_CAPACITY, ERR_NOMEM, ERR_BUG = 0, 1, -1, -2, -5, -6


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (portable flags only)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "rr_oracle.h"))):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-shared", "-fPIC",
                               _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def load(path: str):
    """Loads an oracle library from `path` and declares its entry points."""
    L = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i32, i64 = ctypes.c_int, ctypes.c_int64
    L.rro_window.argtypes = [P, i32, i32, i32]
    L.rro_window.restype = i32
    L.rro_split.argtypes = [P, i32, P, i32, P, i32, i32, i32, i32, P]
    L.rro_split.restype = i32
    L.rro_plan_mode.argtypes = [P, i32, i32, i32, i32, i32, i32, P, i64, P, P, P, i64, P, i32]
    L.rro_plan_mode.restype = i32
    L.rro_bird_mode.argtypes = [P, i32, i32, i32, i32, i32, i32, P, i64, P, P, i64, P, i32]
    L.rro_bird_mode.restype = i32
    L.rro_bird_prefix.argtypes = [P, i32, i32, i32, i32, i32, i32, P, i64, P, i64]
    L.rro_bird_prefix.restype = i32
    L.rro_batch.argtypes = [P, i64, i32, i32, P, i64, P, i64, P, P]
    L.rro_batch.restype = i32
    L.rro_batch_prefix.argtypes = [P, i64, i32, i32, i64, P, i64, P, i64, P, P]
    L.rro_batch_prefix.restype = i32
    return L


def lib():
    """The oracle library: the one built here, or the one named by
    RR_ORACLE_LIB (the pin-strength test points it at deliberately broken
    copies of the oracle)."""
    global _lib
    if _lib is None:
        _lib = load(os.environ.get("RR_ORACLE_LIB") or build())
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None and a.size else None


def window(s, r0: int, h: int) -> int:
    s = np.ascontiguousarray(s, dtype=np.int32)
    return lib().rro_window(_ptr(s) or ctypes.c_void_p(1), len(s), r0, h) if len(s) else (
        0 if h == 0 else -1)


def split(mand, top, bot, x: int, r0: int, h: int):
    mand = np.ascontiguousarray(mand, dtype=np.int32)
    top = np.ascontiguousarray(top, dtype=np.int32)
    bot = np.ascontiguousarray(bot, dtype=np.int32)
    cost = ctypes.c_int64(0)
    a = lib().rro_split(_ptr(mand), len(mand), _ptr(top), len(top), _ptr(bot), len(bot),
                        x, r0, h, ctypes.byref(cost))
    return a, cost.value


class Plan:
    def __init__(self, status, moves, sigma, events):
        self.status = status
        self.moves = moves          # (k, 4) int32: src_row, src_col, dst_row, dst_col
        self.sigma = sigma          # (n,) int32 surplus after the column phase
        self.events = events        # (e, 5) int32: case, donor, receiver, x, a


def plan(grid: np.ndarray, rect, with_trace: bool = False, strict: bool = False) -> Plan:
    """red-rec (Alg. 1). strict: the strict-reservoir reading of target
    sub-rectangles (outer columns donate reservoir-row atoms only)."""
    grid = np.ascontiguousarray(grid, dtype=np.uint8)
    m, n = grid.shape
    r0, c0, r1, c1 = (int(v) for v in rect)
    nm = ctypes.c_int64(0)
    ne = ctypes.c_int64(0)
    sigma = np.zeros(n, dtype=np.int32)
    cap = 0
    cap_ev = 2 * n + 2 if with_trace else 0
    events = np.zeros((max(cap_ev, 1), 5), dtype=np.int32)
    while True:
        moves = np.zeros((max(cap, 1), 4), dtype=np.int32)
        st = lib().rro_plan_mode(_ptr(grid), m, n, r0, c0, r1, c1, _ptr(moves), cap,
                                 ctypes.byref(nm), _ptr(sigma), _ptr(events) if with_trace else None,
                                 cap_ev, ctypes.byref(ne), int(strict))
        if st == ERR_CAPACITY:
            cap = nm.value
            continue
        break
    if st not in (OK, INFEASIBLE):
        raise RuntimeError(f"oracle rro_plan failed with status {st}")
    return Plan(st, moves[: nm.value].copy(), sigma,
                events[: ne.value].copy() if with_trace else None)


def bird(grid: np.ndarray, rect, with_trace: bool = False, strict: bool = False) -> Plan:
    """The bird planner (Alg. 2, Sec. III.E). With with_trace, events holds
    one row per receiver: (column, tokens from above the band, tokens from
    below it); sigma is not filled. strict as in plan()."""
    grid = np.ascontiguousarray(grid, dtype=np.uint8)
    m, n = grid.shape
    r0, c0, r1, c1 = (int(v) for v in rect)
    nm = ctypes.c_int64(0)
    nu = ctypes.c_int64(0)
    cap = 0
    cap_u = n + 1 if with_trace else 0
    units = np.zeros((max(cap_u, 1), 3), dtype=np.int32)
    while True:
        moves = np.zeros((max(cap, 1), 4), dtype=np.int32)
        st = lib().rro_bird_mode(_ptr(grid), m, n, r0, c0, r1, c1, _ptr(moves), cap, ctypes.byref(nm),
                                 _ptr(units) if with_trace else None, cap_u, ctypes.byref(nu), int(strict))
        if st == ERR_CAPACITY:
            cap = nm.value
            continue
        break
    if st not in (OK, INFEASIBLE):
        raise RuntimeError(f"oracle rro_bird failed with status {st}")
    return Plan(st, moves[: nm.value].copy(), None, units[: nu.value].copy() if with_trace else None)


def bird_prefix(grid: np.ndarray, rect, max_units: int) -> Plan:
    """The bird planner stopped after its first max_units receiver units."""
    grid = np.ascontiguousarray(grid, dtype=np.uint8)
    m, n = grid.shape
    r0, c0, r1, c1 = (int(v) for v in rect)
    nm = ctypes.c_int64(0)
    cap = 0
    while True:
        moves = np.zeros((max(cap, 1), 4), dtype=np.int32)
        st = lib().rro_bird_prefix(_ptr(grid), m, n, r0, c0, r1, c1, _ptr(moves), cap, ctypes.byref(nm),
                                   int(max_units))
        if st == ERR_CAPACITY:
            cap = nm.value
            continue
        break
    if st not in (OK, INFEASIBLE):
        raise RuntimeError(f"oracle rro_bird_prefix failed with status {st}")
    return Plan(st, moves[: nm.value].copy(), None, None)


def batch(moves: np.ndarray, m: int, n: int, max_ops: int | None = None, cap: int = 0):
    """Returns (ops (b, 3) int32: dir, first, count; members (s,) int32).
    With max_ops, only the first max_ops batches. cap: initial room for ops
    and members (a caller that knows the total path length passes it and
    the routine runs once instead of sizing first)."""
    moves = np.ascontiguousarray(moves, dtype=np.int32).reshape(-1, 4)
    no = ctypes.c_int64(0)
    nmem = ctypes.c_int64(0)
    cap_o = cap_m = int(cap)
    while True:
        ops = np.zeros((max(cap_o, 1), 3), dtype=np.int32)
        mem = np.zeros(max(cap_m, 1), dtype=np.int32)
        if max_ops is None:
            st = lib().rro_batch(_ptr(moves), len(moves), m, n, _ptr(ops), cap_o, _ptr(mem), cap_m,
                                 ctypes.byref(no), ctypes.byref(nmem))
        else:
            st = lib().rro_batch_prefix(_ptr(moves), len(moves), m, n, int(max_ops), _ptr(ops), cap_o,
                                        _ptr(mem), cap_m, ctypes.byref(no), ctypes.byref(nmem))
        if st == ERR_CAPACITY:
            cap_o, cap_m = no.value, nmem.value
            continue
        break
    if st != OK:
        raise RuntimeError(f"oracle rro_batch failed with status {st}")
    return ops[: no.value].copy(), mem[: nmem.value].copy()
