"""Writes tests/golden/digests/oracle_1024.json: SHA-256 digests of the oracle's
complete outputs on the 1024 x 1024 workload (fill 0.6, centred 720 x 720
target, seed 0, grid 0), for outputs too large to recompute inside a test.

Only the oracle (oracle/) and the seeded input generator (gridgen/) are
called. A digest is the SHA-256 of the little-endian int32 array bytes, C
order: moves (k, 4) = (src_row, src_col, dst_row, dst_col); ops (b, 3) =
(dir, first, count); members (s,). Batching the red-rec plan takes the
oracle about ten minutes on one core (46.9 M batches, Alg. 4 taken
literally); the bird plan about as long again.

    python tests/golden/digests/make_digests.py [--no-bird]
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(os.path.dirname(HERE)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import gridgen  # noqa: E402
import oracle  # noqa: E402

OUT = os.path.join(HERE, "oracle_1024.json")


def sha(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a, dtype="<i4").tobytes()).hexdigest()


def entry(plan, m, n):
    t0 = time.time()
    ops, mem = oracle.batch(plan.moves, m, n)
    return {
        "status": int(plan.status),
        "n_moves": int(len(plan.moves)),
        "n_ops": int(len(ops)),
        "n_members": int(len(mem)),
        "moves_sha256": sha(plan.moves),
        "ops_sha256": sha(ops),
        "members_sha256": sha(mem),
        "oracle_batch_seconds": round(time.time() - t0, 1),
    }


def main():
    inst = gridgen.square_instance(0, 0, 1024, 0.6, 720)
    out = {
        "workload": "1024 x 1024, Bernoulli(0.6) from gridgen.square_instance(seed 0, grid 0), "
                    "centred 720 x 720 target",
        "rect": list(inst.rect),
        "written_by": "tests/golden/digests/make_digests.py (oracle only)",
    }
    out["redrec"] = entry(oracle.plan(inst.grid, inst.rect), 1024, 1024)
    print("red-rec", out["redrec"], flush=True)
    if "--no-bird" not in sys.argv:
        out["bird"] = entry(oracle.bird(inst.grid, inst.rect), 1024, 1024)
        print("bird", out["bird"], flush=True)
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
