"""The oracle built with the address and undefined-behaviour sanitizers runs
red-rec, bird (both readings of target sub-rectangles) and the batching
routine on random grids of odd shapes and on 128 x 128 grids without a
report: no out-of-bounds access, use after free or undefined arithmetic in
the code that defines the expected results. (CPU only; skipped where the
compiler has no sanitizer runtime.)"""
import os
import subprocess
import sys
import textwrap

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

SCRIPT = textwrap.dedent("""
    import sys
    sys.path.insert(0, {root!r})
    import numpy as np
    import gridgen, oracle
    assert oracle.lib()._name == {lib!r}
    for seed in range(2):
        i = gridgen.square_instance(seed, 0, 128, 0.6)
        for strict in (False, True):
            for planner in (oracle.plan, oracle.bird):
                p = planner(i.grid, i.rect, strict=strict)
                if p.status == 0:
                    oracle.batch(p.moves, 128, 128)
    rng = np.random.default_rng(11)
    for t in range(150):
        m, n = (int(v) for v in rng.integers(1, 40, 2))
        g = (rng.random((m, n)) < rng.uniform(0.2, 0.95)).astype(np.uint8)
        r0 = int(rng.integers(0, m)); r1 = int(rng.integers(r0 + 1, m + 1))
        c0 = int(rng.integers(0, n)); c1 = int(rng.integers(c0 + 1, n + 1))
        for strict in (False, True):
            for planner in (oracle.plan, oracle.bird):
                p = planner(g, (r0, c0, r1, c1), strict=strict)
                if p.status == 0:
                    oracle.batch(p.moves, m, n)
    print("sanitized oracle ok")
""")


def _runtime(name):
    p = subprocess.run(["gcc", f"-print-file-name={name}"], capture_output=True, text=True)
    path = p.stdout.strip()
    return path if p.returncode == 0 and os.path.isabs(path) and os.path.exists(path) else None


def test_oracle_under_address_and_ub_sanitizers(tmp_path):
    asan, ubsan = _runtime("libasan.so"), _runtime("libubsan.so")
    if not asan or not ubsan:
        pytest.skip("no sanitizer runtime for the host compiler")
    lib = str(tmp_path / "liboracle_san.so")
    subprocess.check_call(["gcc", "-O1", "-g", "-std=c11", "-shared", "-fPIC", "-fno-omit-frame-pointer",
                           "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined",
                           os.path.join(ROOT, "oracle", "rr_oracle.c"), "-o", lib])
    env = dict(os.environ, LD_PRELOAD=f"{asan} {ubsan}", RR_ORACLE_LIB=lib,
               ASAN_OPTIONS="detect_leaks=0:halt_on_error=1", UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    p = subprocess.run([sys.executable, "-c", SCRIPT.format(root=ROOT, lib=lib)], env=env, capture_output=True,
                       text=True, timeout=600)
    out = p.stdout + p.stderr
    assert p.returncode == 0, out[-3000:]
    assert "sanitized oracle ok" in p.stdout
    assert "runtime error" not in out and "AddressSanitizer" not in out, out[-3000:]
