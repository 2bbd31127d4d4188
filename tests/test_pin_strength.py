"""Strength of the oracle's pins: plausible mistakes, planted one at a time
in a scratch copy of the oracle (never in the oracle itself), must each make
the CPU pin suite fail, and the unmodified copy must pass it.

Each mutant is a one-line change of the kind the pins exist to catch: a
wrong sign or index, a flipped tie rule, a dropped condition, an off-by-one
bound. The pin suite runs in a child pytest process with RR_ORACLE_LIB
pointing at the mutant's library."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "rr_oracle.c")
PINS = ["tests/test_oracle_golden.py", "tests/test_oracle_pins.py", "tests/test_oracle_batching.py",
        "tests/test_oracle_bird.py", "tests/test_oracle_strict.py"]

# (name, text, replacement, which occurrence)
MUTANTS = [
    ("bird_top_projection_sign", "else if (r < r0) T[nt++] = (btok_t){r - d, r, c};",
     "else if (r < r0) T[nt++] = (btok_t){r + d, r, c};", 0),
    ("bird_bottom_projection_sign", "else if (r >= r1) T[nt++] = (btok_t){r + d, r, c};",
     "else if (r >= r1) T[nt++] = (btok_t){r - d, r, c};", 0),
    ("bird_farthest_token_of_vertex", "if (pos[k] < r0) for (int q = g1 - want; q < g1; ++q) take[q] = 1;",
     "if (pos[k] < r0) for (int q = g0; q < g0 + want; ++q) take[q] = 1;", 0),
    ("bird_right_before_left", "if (ra != rb) return ra ? -1 : 1;", "if (ra != rb) return ra ? 1 : -1;", 1),
    ("window_largest_start_on_ties", "if (c < bc) { bc = c; best = w; }", "if (c <= bc) { bc = c; best = w; }", 0),
    ("split_smallest_a_on_ties", "if (best < 0 || c <= bc) { bc = c; best = a; }",
     "if (best < 0 || c < bc) { bc = c; best = a; }", 0),
    ("emission_downward_shallowest_first", "for (int k = cnt - 1; k >= 0; --k)", "for (int k = 0; k < cnt; ++k)", 0),
    ("projected_row_ties_right_first_below", "if (ra != rb) return ra ? 1 : -1;", "if (ra != rb) return ra ? -1 : 1;", 0),
    ("outer_virtual_targets_reversed", "for (int k = 0; k < r0; ++k) unit[cnt++] = (mv_t){s[k], c, k, c};",
     "for (int k = 0; k < r0; ++k) unit[cnt++] = (mv_t){s[k], c, r0 - 1 - k, c};", 0),
    ("pairing_prefers_larger_gap", "else if (d != bd) better = d < bd;", "else if (d != bd) better = d > bd;", 0),
    ("feasibility_off_by_one", "if (tot < 0) { st = INFEASIBLE; out.n = 0; goto done; }",
     "if (tot < -1) { st = INFEASIBLE; out.n = 0; goto done; }", 0),
    ("batch_without_same_line", "ok = accr[a] == r || accc[a] == c;", "ok = 1;", 0),
    ("batch_without_same_direction", "ok = d == d0;", "ok = 1;", 0),
    ("gamma_ignores_shared_vertices", "if (cover[off[v]] != b) blocked[b]++;", "if (0) blocked[b]++;", 0),
    ("bird_receivers_right_to_left", "for (int j = c0; j < c1; ++j) {", "for (int j = c1 - 1; j >= c0; --j) {", 0),
    ("strict_mode_ignored_in_redrec", "} else if (!strict && K[c] >= R) {", "} else if (K[c] >= R) {", 0),
    ("strict_mode_ignored_in_bird", "} else if (!strict && K >= R) {", "} else if (K >= R) {", 0),
    ("bird_skips_unsolved_columns", "if (c == j) T[nt++] = (btok_t){r, r, c};",
     "if (c == j) T[nt++] = (btok_t){r, r, c};\n                else if (recv[c]) continue;", 0),
]


def _build(tmp, name, text):
    src = os.path.join(tmp, name + ".c")
    lib = os.path.join(tmp, name + ".so")
    with open(src, "w") as f:
        f.write(text)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-I", os.path.join(ROOT, "oracle"),
                           src, "-o", lib])
    return lib


def _pins_pass(lib):
    env = dict(os.environ, RR_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PINS],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    return r.returncode == 0


def _mutate(text, old, new, occurrence):
    at = -1
    for _ in range(occurrence + 1):
        at = text.index(old, at + 1)
    return text[:at] + new + text[at + len(old):]


def test_unmodified_copy_passes(tmp_path):
    assert _pins_pass(_build(str(tmp_path), "control", open(SRC).read()))


@pytest.mark.parametrize("name,old,new,occ", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(tmp_path, name, old, new, occ):
    text = open(SRC).read()
    assert text.count(old) >= occ + 1, f"anchor of {name} not found"
    mutant = _mutate(text, old, new, occ)
    assert mutant != text
    assert not _pins_pass(_build(str(tmp_path), name, mutant)), f"no pin catches {name}"
