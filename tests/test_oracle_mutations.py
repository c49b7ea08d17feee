"""Planted mistakes in the oracle: each one must fail a pin.

Each case copies oracle/bc_oracle.c, changes one expression (a dropped term,
a transposed operand, a wrong index or bound), builds the copy into a
temporary library with the oracle's compiler flags, and runs the pins of
tests/test_oracle_pins.py against it in a child process (the child points
the oracle package at the temporary library before the pins import it).
Every planted mistake must make a pin fail; an unchanged copy built the same
way must pass them all, so a failure means the pins saw the mistake and not
a broken harness. The mistakes live only in the temporary copies.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "bc_oracle.c")
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")

# (name, expression in bc_oracle.c, planted replacement); each expression occurs once
MUTANTS = [
    ("eq4_dropped_one", "double coef = (1.0 + ws->delta[x]);", "double coef = (ws->delta[x]);"),
    ("eq4_sigma_ratio_transposed", "ws->delta[v] += ws->sigma[v] / ws->sigma[x] * coef;",
     "ws->delta[v] += ws->sigma[x] / ws->sigma[v] * coef;"),
    ("rv_keeps_r", "if (seen[v] && v != r)", "if (seen[v])"),
    ("philox_wrong_key_word", "c0 = hi1 ^ c1 ^ k0;", "c0 = hi1 ^ c1 ^ k1;"),
    ("approx_scale_off_by_one", "double scale = (double)k / (double)T;",
     "double scale = (double)k / (double)(T + 1);"),
    ("sigma_skips_first_settled", "for (int64_t i = 1; i < k; i++) {", "for (int64_t i = 2; i < k; i++) {"),
    ("prop1_wrong_degree_test", "if (out_degree(off, r) == 0) return 0.0;",
     "if (out_degree(off, r) <= 1) return 0.0;"),
    ("dijkstra_ignores_weights", "uint64_t nd = dx + (uint64_t)g->w[e];", "uint64_t nd = dx + 1;"),
    ("reverse_graph_drops_weights", "if (w && rw) rw[p] = w[e];", "if (w && rw) rw[p] = 1;"),
    ("bfs_step_of_two", "ws->dist[y] = ws->dist[x] + 1;", "ws->dist[y] = ws->dist[x] + 2;"),
    ("approx_drops_multiplicity", "for (int64_t t = 0; t < T; t++) bc += dep[slot[draw[t]]] * scale;",
     "for (int64_t t = 0; t < nu; t++) bc += dep[t] * scale;"),
    ("sample_index_modulo", "return (int64_t)(((u128)out[0] * (u128)(uint64_t)k) >> 64);",
     "return (int64_t)(out[0] % (uint64_t)k);"),
]

RUNNER = """
import sys
import pytest
sys.path[:0] = [{root!r}]
import oracle
oracle._build.build = lambda force=False: {lib!r}
sys.exit(pytest.main(["-q", "-x", "-p", "no:cacheprovider", {pins!r}]))
"""


def build_variant(tmp_path, old=None, new=None):
    with open(SRC) as f:
        src = f.read()
    if old is not None:
        assert src.count(old) == 1, old
        src = src.replace(old, new)
    c = tmp_path / "variant.c"
    c.write_text(src)
    so = tmp_path / "libvariant.so"
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-pthread", "-w", str(c), "-o", str(so)])
    return str(so)


def run_pins(lib):
    code = RUNNER.format(root=ROOT, lib=lib, pins=PINS)
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=900)
    return r.returncode, (r.stdout + r.stderr)[-3000:]


def test_unchanged_copy_passes(tmp_path):
    rc, out = run_pins(build_variant(tmp_path))
    assert rc == 0, out


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(tmp_path, name, old, new):
    rc, out = run_pins(build_variant(tmp_path, old, new))
    assert rc == 1, (name, rc, out)  # 1: a pin failed (not a crash, a usage error or no tests)
