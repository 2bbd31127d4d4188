"""The stored digests of the oracle's complete 1024 x 1024 outputs
(tests/golden/digests/oracle_1024.json) belong to the oracle as it stands: the
red-rec move list is replanned here and hashed (the batch digests take the
oracle minutes and are checked against the GPU in the -m gpu tests), and the
counts are consistent with the moves they describe."""
import hashlib
import json
import os

import numpy as np

import gridgen
import oracle


def _gold():
    with open(os.path.join(os.path.dirname(__file__), "golden", "digests", "oracle_1024.json")) as f:
        return json.load(f)


def test_redrec_move_digest_is_the_oracles():
    gold = _gold()
    inst = gridgen.square_instance(0, 0, 1024, 0.6, 720)
    assert list(inst.rect) == gold["rect"]
    ref = oracle.plan(inst.grid, inst.rect)
    g = gold["redrec"]
    assert ref.status == g["status"] == 0 and len(ref.moves) == g["n_moves"]
    assert hashlib.sha256(np.ascontiguousarray(ref.moves, dtype="<i4").tobytes()).hexdigest() == g["moves_sha256"]
    steps = int((np.abs(ref.moves[:, 0] - ref.moves[:, 2]) + np.abs(ref.moves[:, 1] - ref.moves[:, 3])).sum())
    assert steps == g["n_members"]              # every elementary step is one batch member (Alg. 4)
    assert g["n_ops"] <= g["n_members"]


def test_bird_counts_are_consistent():
    g = _gold()["bird"]
    assert g["status"] == 0 and g["n_ops"] <= g["n_members"]
    assert len(g["moves_sha256"]) == len(g["ops_sha256"]) == len(g["members_sha256"]) == 64
