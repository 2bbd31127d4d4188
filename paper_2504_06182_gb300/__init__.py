"""GB300 red-rec planner and batching routine (arXiv 2504.06182, Alg. 1 and
Alg. 4) -- Python binding of the C ABI in include/rr.h.

The functions below carry the C names and only marshal arguments: every step
of the planning and batching path runs in the CUDA library librr.so. PyTorch
is used for device memory and streams. If librr.so is missing the import of
the binding fails loudly; nothing falls back to a CPU path.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librr.so")

RR_OK, RR_INFEASIBLE = 0, 1
RR_ERR_ARG, RR_ERR_CAPACITY, RR_ERR_CUDA = -1, -2, -3
RR_ERR_TIMEOUT, RR_ERR_WORKSPACE, RR_ERR_INTERNAL = -4, -5, -6
RR_U8, RR_BITS32 = 0, 1
RR_WITH_BATCH = 1
RR_BATCH_ONLY = 2
RR_GRAPH = 4
RR_BIRD = 8
RR_STRICT_RESERVOIR = 16
RR_MAX_SIDE = 1024
STATUS_NAMES = {0: "OK", 1: "INFEASIBLE", -1: "ERR_ARG", -2: "ERR_CAPACITY", -3: "ERR_CUDA",
                -4: "ERR_TIMEOUT", -5: "ERR_WORKSPACE", -6: "ERR_INTERNAL"}


class rr_rect(ctypes.Structure):
    _fields_ = [("r0", ctypes.c_int32), ("c0", ctypes.c_int32), ("r1", ctypes.c_int32), ("c1", ctypes.c_int32)]


class rr_move(ctypes.Structure):
    _fields_ = [("src_row", ctypes.c_int32), ("src_col", ctypes.c_int32),
                ("dst_row", ctypes.c_int32), ("dst_col", ctypes.c_int32)]


class rr_op(ctypes.Structure):
    _fields_ = [("dir", ctypes.c_int32), ("first", ctypes.c_int32), ("count", ctypes.c_int32)]


class rr_instance(ctypes.Structure):
    _fields_ = [("grid", ctypes.c_void_p), ("layout", ctypes.c_int32), ("m", ctypes.c_int32),
                ("n", ctypes.c_int32), ("pad0", ctypes.c_int32), ("rect", rr_rect),
                ("moves", ctypes.c_void_p), ("cap_moves", ctypes.c_int64),
                ("ops", ctypes.c_void_p), ("cap_ops", ctypes.c_int64),
                ("members", ctypes.c_void_p), ("cap_members", ctypes.c_int64),
                ("n_moves", ctypes.c_int64), ("n_steps", ctypes.c_int64),
                ("n_ops", ctypes.c_int64), ("n_members", ctypes.c_int64),
                ("status", ctypes.c_int32), ("pad1", ctypes.c_int32)]


class rr_serve_config(ctypes.Structure):
    _fields_ = [("max_side", ctypes.c_int32), ("slots", ctypes.c_int32), ("streams", ctypes.c_int32),
                ("max_wave", ctypes.c_int32), ("flags", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("arena_bytes", ctypes.c_int64), ("heap_bytes", ctypes.c_int64), ("input_bytes", ctypes.c_int64)]


class rr_serve_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("m", ctypes.c_int32), ("n", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("n_moves", ctypes.c_int64), ("n_steps", ctypes.c_int64), ("n_ops", ctypes.c_int64),
                ("n_members", ctypes.c_int64), ("d_moves", ctypes.c_void_p), ("d_ops", ctypes.c_void_p),
                ("d_members", ctypes.c_void_p), ("t_submit_us", ctypes.c_double), ("t_admit_us", ctypes.c_double),
                ("t_done_us", ctypes.c_double)]


EXPORTS = ("rr_ctx_create", "rr_ctx_destroy", "rr_plan", "rr_bird_plan", "rr_plan_mode", "rr_batch", "rr_plan_batched", "rr_set_tracing",
           "rr_stage_times", "rr_launch_count", "rr_autotune", "rr_set_config", "rr_last_error", "rr_plan_noalloc", "rr_plan_one", "rr_debug_guard_limit", "rr_serve_open", "rr_serve_submit",
           "rr_serve_poll", "rr_serve_release", "rr_serve_close")
RR_NOALLOC_MAX_SIDE = 256
RR_ONE_MAX_SIDE = 256

_lib = None


def load(path: str = LIB_PATH):
    """Load librr.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing: build it with paper_2504_06182_gb300.build.build()")
    L = ctypes.CDLL(path)
    P, I32, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    L.rr_ctx_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), I64]
    L.rr_ctx_create.restype = I32
    L.rr_ctx_destroy.argtypes = [P]
    L.rr_ctx_destroy.restype = I32
    L.rr_plan.argtypes = [P, P, I32, I32, I32, rr_rect, P, I64, ctypes.POINTER(I64), P]
    L.rr_plan.restype = I32
    L.rr_bird_plan.argtypes = [P, P, I32, I32, I32, rr_rect, P, I64, ctypes.POINTER(I64), P]
    L.rr_bird_plan.restype = I32
    L.rr_plan_mode.argtypes = [P, P, I32, I32, I32, rr_rect, I32, P, I64, ctypes.POINTER(I64), P]
    L.rr_plan_mode.restype = I32
    L.rr_batch.argtypes = [P, P, I64, I32, I32, P, I64, P, I64, ctypes.POINTER(I64), ctypes.POINTER(I64), P]
    L.rr_batch.restype = I32
    L.rr_plan_batched.argtypes = [P, P, I32, I32, I32, P]
    L.rr_plan_batched.restype = I32
    L.rr_set_tracing.argtypes = [P, I32]
    L.rr_set_tracing.restype = I32
    L.rr_stage_times.argtypes = [P, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_char_p), I32]
    L.rr_stage_times.restype = I32
    L.rr_launch_count.argtypes = [P, ctypes.POINTER(ctypes.c_int64)]
    L.rr_launch_count.restype = I32
    L.rr_autotune.argtypes = [P, P, I32, I32, I32, P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                              ctypes.POINTER(ctypes.c_int32)]
    L.rr_autotune.restype = I32
    L.rr_set_config.argtypes = [P, I32, I32, I32]
    L.rr_set_config.restype = I32
    L.rr_plan_noalloc.argtypes = [P, I32, I32, I32, rr_rect, P, I64, ctypes.POINTER(I64), P]
    L.rr_plan_noalloc.restype = I32
    L.rr_plan_one.argtypes = [P, P, I32, I32, I32, rr_rect, I32, P, I64, P, I64, P, I64, ctypes.POINTER(I64), P]
    L.rr_plan_one.restype = I32
    L.rr_debug_guard_limit.argtypes = [I64]
    L.rr_debug_guard_limit.restype = I32
    L.rr_serve_open.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(rr_serve_config)]
    L.rr_serve_open.restype = I32
    L.rr_serve_submit.argtypes = [P, P, I32, I32, I32, rr_rect, ctypes.POINTER(I64)]
    L.rr_serve_submit.restype = I32
    L.rr_serve_poll.argtypes = [P, I64, ctypes.POINTER(rr_serve_result), I64]
    L.rr_serve_poll.restype = I32
    L.rr_serve_release.argtypes = [P, I64]
    L.rr_serve_release.restype = I32
    L.rr_serve_close.argtypes = [P]
    L.rr_serve_close.restype = I32
    L.rr_last_error.argtypes = [P]
    L.rr_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def _addr(x) -> int:
    """Device address of a torch tensor, or an integer address as is."""
    if x is None:
        return 0
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    return int(x)


def _stream(stream) -> int:
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return int(stream.cuda_stream)
    return int(stream)


class RRError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


# ------------------------------------------------------------- C-ABI names

def rr_ctx_create(arena_bytes: int = 0) -> int:
    h = ctypes.c_void_p(0)
    st = load().rr_ctx_create(ctypes.byref(h), int(arena_bytes))
    if st != RR_OK:
        raise RRError(st, load().rr_last_error(None).decode())
    return h.value


def rr_ctx_destroy(ctx: int) -> int:
    return load().rr_ctx_destroy(ctx)


def rr_last_error(ctx) -> str:
    return load().rr_last_error(ctx).decode()


def rr_plan(ctx, d_grid, layout, m, n, rect, d_moves, cap, stream=None):
    """Returns (status, n_moves)."""
    nm = ctypes.c_int64(0)
    st = load().rr_plan(ctx, _addr(d_grid), int(layout), int(m), int(n), rr_rect(*[int(v) for v in rect]),
                        _addr(d_moves), int(cap), ctypes.byref(nm), _stream(stream))
    return st, nm.value


def rr_bird_plan(ctx, d_grid, layout, m, n, rect, d_moves, cap, stream=None):
    """The bird planner (Alg. 2, Sec. III.E). Returns (status, n_moves)."""
    nm = ctypes.c_int64(0)
    st = load().rr_bird_plan(ctx, _addr(d_grid), int(layout), int(m), int(n), rr_rect(*[int(v) for v in rect]),
                             _addr(d_moves), int(cap), ctypes.byref(nm), _stream(stream))
    return st, nm.value


def rr_plan_mode(ctx, d_grid, layout, m, n, rect, flags, d_moves, cap, stream=None):
    """Planning with flags RR_BIRD / RR_STRICT_RESERVOIR. Returns (status, n_moves)."""
    nm = ctypes.c_int64(0)
    st = load().rr_plan_mode(ctx, _addr(d_grid), int(layout), int(m), int(n), rr_rect(*[int(v) for v in rect]),
                             int(flags), _addr(d_moves), int(cap), ctypes.byref(nm), _stream(stream))
    return st, nm.value


def rr_batch(ctx, d_moves, n_moves, m, n, d_ops, cap_ops, d_members, cap_members, stream=None):
    """Returns (status, n_ops, n_members)."""
    no, nmem = ctypes.c_int64(0), ctypes.c_int64(0)
    st = load().rr_batch(ctx, _addr(d_moves), int(n_moves), int(m), int(n), _addr(d_ops), int(cap_ops),
                         _addr(d_members), int(cap_members), ctypes.byref(no), ctypes.byref(nmem),
                         _stream(stream))
    return st, no.value, nmem.value


def rr_plan_batched(ctx, d_inst, count, max_side, flags=0, stream=None) -> int:
    return load().rr_plan_batched(ctx, _addr(d_inst), int(count), int(max_side), int(flags), _stream(stream))


def rr_set_tracing(ctx, enable: bool) -> int:
    return load().rr_set_tracing(ctx, 1 if enable else 0)


def rr_stage_times(ctx, cap: int = 32):
    """[(kernel name, ms)] of the most recent traced call."""
    ms = (ctypes.c_float * cap)()
    names = (ctypes.c_char_p * cap)()
    k = load().rr_stage_times(ctx, ms, names, cap)
    if k < 0:
        raise RRError(k, rr_last_error(ctx))
    return [(names[i].decode(), float(ms[i])) for i in range(k)]


def rr_autotune(ctx, d_inst, count, max_side, flags=RR_WITH_BATCH, stream=None):
    """Picks and keeps the fastest launch configuration for these instances.
    Returns (size classes, log2 block-budget scale, pipeline split 0..4)."""
    nc, sh, pd = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
    st = load().rr_autotune(ctx, _addr(d_inst), int(count), int(max_side), int(flags), _stream(stream),
                            ctypes.byref(nc), ctypes.byref(sh), ctypes.byref(pd))
    if st != RR_OK:
        raise RRError(st, rr_last_error(ctx))
    return int(nc.value), int(sh.value), int(pd.value)


def rr_set_config(ctx, nclass, shift, pipe) -> int:
    """Sets the batched launch configuration (size classes, log2 block-budget
    scale, pipeline split)."""
    st = load().rr_set_config(ctx, int(nclass), int(shift), int(pipe))
    if st != RR_OK:
        raise RRError(st, rr_last_error(ctx))
    return st


def rr_launch_count(ctx) -> int:
    """Kernels the context has launched since it was created."""
    v = ctypes.c_int64(0)
    st = load().rr_launch_count(ctx, ctypes.byref(v))
    if st != RR_OK:
        raise RRError(st, rr_last_error(ctx))
    return int(v.value)


def rr_plan_noalloc(d_grid, layout, m, n, rect, d_moves, cap, stream=None):
    """rr_plan without a context or any allocation (sides up to
    RR_NOALLOC_MAX_SIDE). Returns (status, n_moves)."""
    nm = ctypes.c_int64(0)
    st = load().rr_plan_noalloc(_addr(d_grid), int(layout), int(m), int(n), rr_rect(*[int(v) for v in rect]),
                                _addr(d_moves), int(cap), ctypes.byref(nm), _stream(stream))
    return st, nm.value


def rr_plan_one(ctx, d_grid, layout, m, n, rect, flags, d_moves, cap_moves, d_ops=None, cap_ops=0, d_members=None,
                cap_members=0, stream=None):
    """Plan (and with RR_WITH_BATCH batch) one grid in one kernel launch.
    Returns (status, n_moves, n_steps, n_ops, n_members)."""
    counts = (ctypes.c_int64 * 4)()
    st = load().rr_plan_one(ctx, _addr(d_grid), int(layout), int(m), int(n), rr_rect(*[int(v) for v in rect]),
                            int(flags), _addr(d_moves), int(cap_moves), _addr(d_ops), int(cap_ops), _addr(d_members),
                            int(cap_members), counts, _stream(stream))
    return (st, *[int(c) for c in counts])


def rr_debug_guard_limit(limit: int) -> int:
    """Caps the pairing loop and the batching simulation at `limit`
    iterations (0: the built-in bounds), for tests of the timeout path."""
    return load().rr_debug_guard_limit(int(limit))


# ------------------------------------------------------------------ serving

def rr_serve_open(max_side, slots, streams, max_wave, flags=RR_WITH_BATCH, arena_bytes=0, heap_bytes=1 << 30,
                  input_bytes=0):
    cfg = rr_serve_config(int(max_side), int(slots), int(streams), int(max_wave), int(flags), 0,
                          int(arena_bytes), int(heap_bytes), int(input_bytes))
    h = ctypes.c_void_p(0)
    st = load().rr_serve_open(ctypes.byref(h), ctypes.byref(cfg))
    if st != RR_OK:
        raise RRError(st, "rr_serve_open failed")
    return h.value


def rr_serve_submit(srv, h_grid, layout, m, n, rect):
    """h_grid: a contiguous numpy array in host memory. Returns (status, ticket)."""
    t = ctypes.c_int64(0)
    st = load().rr_serve_submit(srv, h_grid.ctypes.data_as(ctypes.c_void_p), int(layout), int(m), int(n),
                                rr_rect(*[int(v) for v in rect]), ctypes.byref(t))
    return st, t.value


def rr_serve_poll(srv, ticket, timeout_us=0):
    """Returns (status, rr_serve_result)."""
    r = rr_serve_result()
    st = load().rr_serve_poll(srv, int(ticket), ctypes.byref(r), int(timeout_us))
    return st, r


def rr_serve_release(srv, ticket) -> int:
    return load().rr_serve_release(srv, int(ticket))


def rr_serve_close(srv) -> int:
    return load().rr_serve_close(srv)
