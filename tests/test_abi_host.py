"""Host-side behaviour of the C ABI that needs no GPU: every entry point
refuses bad arguments with RR_ERR_ARG before touching the device and leaves
a message for rr_last_error; without a device, context creation fails with
RR_ERR_CUDA (there is no CPU fallback); the binding refuses to run without
its library."""
import ctypes

import pytest

import paper_2504_06182_gb300 as rr
from paper_2504_06182_gb300 import build

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    return rr.load(build.build())


def _err(L):
    return L.rr_last_error(None).decode()


def test_entry_points_refuse_null_contexts(L):
    rect = rr.rr_rect(0, 0, 4, 4)
    n = ctypes.c_int64(0)
    grid = ctypes.c_void_p(1)          # never dereferenced: the context check comes first
    assert L.rr_plan(None, grid, rr.RR_U8, 4, 4, rect, None, 0, ctypes.byref(n), None) == rr.RR_ERR_ARG
    assert "rr_plan" in _err(L)
    assert L.rr_bird_plan(None, grid, rr.RR_U8, 4, 4, rect, None, 0, ctypes.byref(n), None) == rr.RR_ERR_ARG
    assert "rr_bird_plan" in _err(L)
    assert L.rr_plan_mode(None, grid, rr.RR_U8, 4, 4, rect, 0, None, 0, ctypes.byref(n), None) == rr.RR_ERR_ARG
    assert "rr_plan_mode" in _err(L)
    no, nm = ctypes.c_int64(0), ctypes.c_int64(0)
    assert L.rr_batch(None, None, 0, 4, 4, None, 0, None, 0, ctypes.byref(no), ctypes.byref(nm), None) == rr.RR_ERR_ARG
    assert "rr_batch" in _err(L)
    assert L.rr_plan_batched(None, None, 1, 32, 0, None) == rr.RR_ERR_ARG
    assert "rr_plan_batched" in _err(L)
    a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    assert L.rr_autotune(None, None, 1, 32, 0, None, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)) == rr.RR_ERR_ARG
    assert L.rr_set_config(None, 4, 0, 1) == rr.RR_ERR_ARG
    assert L.rr_set_tracing(None, 1) == rr.RR_ERR_ARG
    cnt = ctypes.c_int64(0)
    assert L.rr_launch_count(None, ctypes.byref(cnt)) == rr.RR_ERR_ARG
    assert L.rr_ctx_destroy(None) == rr.RR_ERR_ARG
    assert L.rr_plan_noalloc(grid, rr.RR_U8, 0, 4, rect, None, 0, ctypes.byref(n), None) == rr.RR_ERR_ARG


def test_unknown_flags_and_bad_shapes_are_refused(L):
    if torch.cuda.is_available():
        pytest.skip("checks the argument path only where no device can be reached")
    # the flag and size checks come before any device work, whatever the context
    n = ctypes.c_int64(0)
    rect = rr.rr_rect(0, 0, 4, 4)
    assert L.rr_plan_mode(None, ctypes.c_void_p(1), rr.RR_U8, 4, 4, rect, 1 << 20, None, 0, ctypes.byref(n),
                          None) == rr.RR_ERR_ARG
    bad = rr.rr_rect(3, 0, 2, 4)       # r0 >= r1
    assert L.rr_plan_mode(None, ctypes.c_void_p(1), rr.RR_U8, 4, 4, bad, 0, None, 0, ctypes.byref(n),
                          None) == rr.RR_ERR_ARG


def test_serving_refuses_bad_configurations(L):
    h = ctypes.c_void_p(0)
    cfg = rr.rr_serve_config(0, 8, 2, 4, rr.RR_WITH_BATCH, 0, 0, 1 << 20, 0)      # max_side 0
    assert L.rr_serve_open(ctypes.byref(h), ctypes.byref(cfg)) == rr.RR_ERR_ARG
    cfg = rr.rr_serve_config(64, 8, 2, 4, 1 << 20, 0, 0, 1 << 20, 0)               # unknown flag
    assert L.rr_serve_open(ctypes.byref(h), ctypes.byref(cfg)) == rr.RR_ERR_ARG
    assert L.rr_serve_open(None, ctypes.byref(cfg)) == rr.RR_ERR_ARG
    t = ctypes.c_int64(0)
    assert L.rr_serve_submit(None, ctypes.c_void_p(1), rr.RR_U8, 4, 4, rr.rr_rect(0, 0, 4, 4),
                             ctypes.byref(t)) == rr.RR_ERR_ARG
    res = rr.rr_serve_result()
    assert L.rr_serve_poll(None, 0, ctypes.byref(res), 0) == rr.RR_ERR_ARG
    assert L.rr_serve_release(None, 0) == rr.RR_ERR_ARG
    assert L.rr_serve_close(None) == rr.RR_ERR_ARG


def test_no_device_no_fallback(L):
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    with pytest.raises(rr.RRError) as e:
        rr.rr_ctx_create(1 << 20)
    assert e.value.status == rr.RR_ERR_CUDA


def test_binding_refuses_a_missing_library(monkeypatch):
    monkeypatch.setattr(rr, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        rr.load("/nonexistent/librr.so")
