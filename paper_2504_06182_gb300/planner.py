"""Convenience wrapper over the C ABI: a context plus torch-allocated device
buffers. Only buffer management and the capacity protocol of include/rr.h
live here; the planning and batching themselves run in librr.so."""
from __future__ import annotations

import ctypes

import torch

from . import (RR_BIRD, RR_BITS32, RR_ERR_CAPACITY, RR_INFEASIBLE, RR_OK, RR_STRICT_RESERVOIR, RR_U8,
               RR_WITH_BATCH, RRError, rr_batch, rr_ctx_create, rr_ctx_destroy, rr_instance, rr_last_error,
               rr_plan_batched, rr_plan_mode, rr_rect)

INSTANCE_BYTES = ctypes.sizeof(rr_instance)


class Planner:
    def __init__(self, arena_bytes: int = 1 << 30):
        self.ctx = rr_ctx_create(arena_bytes)

    def close(self):
        if self.ctx:
            rr_ctx_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, allowed=(RR_OK,)):
        if st not in allowed:
            raise RRError(st, rr_last_error(self.ctx))

    def plan(self, grid: torch.Tensor, rect, layout: int = RR_U8, n: int | None = None, cap: int | None = None,
             bird: bool = False, strict: bool = False):
        """grid: device tensor, (m, n) uint8 or (m, ceil(n/32)) int32 words.
        bird: plan with the bird algorithm instead of red-rec; strict: the
        strict-reservoir reading of target sub-rectangles.
        Returns (status, moves (k, 4) int32 device tensor)."""
        m = grid.shape[0]
        if n is None:
            n = grid.shape[1] if layout == RR_U8 else grid.shape[1] * 32
        if cap is None:
            cap = max(64, 2 * m * n)
        moves = torch.empty((max(cap, 1), 4), dtype=torch.int32, device=grid.device)
        flags = (RR_BIRD if bird else 0) | (RR_STRICT_RESERVOIR if strict else 0)
        st, k = rr_plan_mode(self.ctx, grid, layout, m, n, rect, flags, moves, cap)
        if st == RR_ERR_CAPACITY:
            return self.plan(grid, rect, layout, n, cap=k, bird=bird, strict=strict)
        self._check(st, (RR_OK, RR_INFEASIBLE))
        return st, moves[:k]

    def batch(self, moves: torch.Tensor, m: int, n: int):
        """Returns (ops (b, 3) int32, members (s,) int32) device tensors."""
        dev = moves.device
        k = moves.shape[0]
        st, nops, nmem = rr_batch(self.ctx, moves, k, m, n, None, 0, None, 0)
        if st == RR_OK:
            return (torch.empty((0, 3), dtype=torch.int32, device=dev),
                    torch.empty((0,), dtype=torch.int32, device=dev))
        if st != RR_ERR_CAPACITY:
            self._check(st)
        ops = torch.empty((max(nops, 1), 3), dtype=torch.int32, device=dev)
        mem = torch.empty((max(nmem, 1),), dtype=torch.int32, device=dev)
        st, nops, nmem = rr_batch(self.ctx, moves, k, m, n, ops, nops, mem, nmem)
        self._check(st)
        return ops[:nops], mem[:nmem]


def pack_instances(entries) -> torch.Tensor:
    """entries: list of dicts with keys grid (device tensor), layout, m, n,
    rect, moves, cap_moves, ops, cap_ops, members, cap_members (tensors or
    None). Returns a device uint8 tensor holding the rr_instance array."""
    arr = (rr_instance * len(entries))()
    for i, e in enumerate(entries):
        x = arr[i]
        x.grid = e["grid"].data_ptr()
        x.layout = e.get("layout", RR_BITS32)
        x.m, x.n = e["m"], e["n"]
        x.rect = rr_rect(*e["rect"])
        for key in ("moves", "ops", "members"):
            t = e.get(key)
            setattr(x, key, t.data_ptr() if t is not None else None)
            setattr(x, "cap_" + key, int(e.get("cap_" + key, 0)))
    raw = torch.frombuffer(bytearray(bytes(arr)), dtype=torch.uint8)
    return raw.to(entries[0]["grid"].device)


def unpack_instances(dev_tensor: torch.Tensor, count: int):
    host = dev_tensor.cpu().numpy().tobytes()
    arr = (rr_instance * count).from_buffer_copy(host)
    return [arr[i] for i in range(count)]


def plan_batched(planner: Planner, inst_tensor: torch.Tensor, count: int, max_side: int, with_batch=True,
                 stream=None, bird=False, strict=False):
    flags = (RR_WITH_BATCH if with_batch else 0) | (RR_BIRD if bird else 0) | (RR_STRICT_RESERVOIR if strict else 0)
    st = rr_plan_batched(planner.ctx, inst_tensor, count, max_side, flags, stream)
    if st != RR_OK:
        raise RRError(st, rr_last_error(planner.ctx))


class _DeviceArray:
    """Exposes a raw device address to torch through __cuda_array_interface__."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3}


def device_view(ptr: int, shape, dtype=torch.int32) -> torch.Tensor:
    """Zero-copy torch view of device memory owned by the library (for
    example a served request's results; valid until the request is
    released)."""
    typestr = {torch.int32: "<i4", torch.uint8: "|u1"}[dtype]
    if not ptr or any(int(d) == 0 for d in shape):
        return torch.empty(tuple(int(d) for d in shape), dtype=dtype, device="cuda")
    return torch.as_tensor(_DeviceArray(ptr, shape, typestr), device="cuda")
