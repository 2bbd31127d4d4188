"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/rr.h (no compute calls: this runs without a GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(rr_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2504_06182_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = declared_functions()
    for want in ("rr_ctx_create", "rr_ctx_destroy", "rr_plan", "rr_batch", "rr_plan_batched"):
        assert want in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if line.strip())
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing


def test_library_loads_via_binding(lib_path):
    import ctypes
    import paper_2504_06182_gb300 as rr
    L = rr.load(lib_path)
    for f in declared_functions():
        assert hasattr(L, f)
    assert ctypes.sizeof(rr.rr_instance) == 128
