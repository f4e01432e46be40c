"""Planted mistakes: each edits a copy of the oracle's C source (on the CPU,
in a temporary folder), compiles it, and checks that at least one pin of
test_oracle_pins fails.  This shows the pins can tell a plausible slip -- a
dropped term, a wrong sign or index, a transposed operand, a strict cap --
from the definition.  Each mutant runs in a child process with a time limit,
since a broken reduction may never terminate (that also counts as caught)."""
import os
import subprocess
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

MUTANTS = [
    ("int d2 drops the square", "acc += (u128)m * (u128)m;", "acc += (u128)m;"),
    ("float d2 drops the running sum", "acc = acc + sq;", "acc = sq;"),
    ("float d2 wrong sign", "(double)pts[(int64_t)i * d + k] - (double)pts[(int64_t)j * d + k]",
     "(double)pts[(int64_t)i * d + k] + (double)pts[(int64_t)j * d + k]"),
    ("integer cap strict", "v <= r2i", "v < r2i"),
    ("float cap strict", "v <= r2)", "v < r2)"),
    ("triangle apex skipped", "k = j + 1; k < n", "k = j + 2; k < n"),
    ("triangle grade ignores one edge", "if (es[ojk].g > g) g = es[ojk].g;", ""),
    ("lex order transposed",
     "  if (p->a != q->a) return p->a < q->a ? -1 : 1;\n  if (p->b != q->b) return p->b < q->b ? -1 : 1;",
     "  if (p->b != q->b) return p->b < q->b ? -1 : 1;\n  if (p->a != q->a) return p->a < q->a ? -1 : 1;"),
    ("face index wrong", "ord[(int64_t)a * n + c],", "ord[(int64_t)a * n + b],"),
    ("faces left unsorted", "if (r[y] < r[x])", "if (0)"),
    ("zero not in the grade set (int)", "  v[m] = 0; /* caller", "  v[m] = m ? v[0] : 0; /* caller"),
    ("zero not in the grade set (float)", "  v[m] = 0.0;", "  v[m] = m ? v[0] : 0.0;"),
    ("edge rows transposed", "out->rowidx[1][2 * t] = es[t].a;", "out->rowidx[1][2 * t] = es[t].b;"),
    ("grade off by one", "eg[t] = (int32_t)find_u128(v, ng, di[t]);",
     "eg[t] = (int32_t)find_u128(v, ng, di[t]) + (di[t] > 0);"),
    ("reduction never adds", "owner[low[j]] = j; }", "}"),
    ("pivot rows not killed", "killed[lowk1[j]] = 1;", ""),
    ("bar endpoints swapped", "b[nb] = gb; e[nb] = gd;", "b[nb] = gd; e[nb] = gb;"),
    ("matrix cap strict", "      if (v <= maxrad) {", "      if (v < maxrad) {"),
    ("tetrahedron apex skipped", "for (int32_t dv = c + 1; dv < n; ++dv)", "for (int32_t dv = c + 2; dv < n; ++dv)"),
    ("tetrahedron grade ignores one edge", "            if (es[ocd].g > g) g = es[ocd].g;\n", ""),
    ("tetrahedron face wrong", "((int64_t)a * nn + c) * nn + dv,", "((int64_t)a * nn + b) * nn + dv,"),
    ("matrix values squared", "if (is_float) df[m] = v;", "if (is_float) df[m] = v * v;"),
]


def _pins():
    """Cheap pins that never reduce a matrix first, then the barcode pins."""
    import test_oracle_pins as P
    for s in range(6):
        yield lambda s=s: P.test_brute_force_tiny(s)
    for s in range(4):
        yield lambda s=s: P.test_dmat_brute_force_tiny(s)
    for s in range(3):
        yield lambda s=s: P.test_tetrahedra_brute_force_tiny(s)
    yield P.test_sortperm_worked_example
    yield P.test_cap_is_inclusive
    yield P.test_float_distance_within_fp64_bound
    for dt in (np.int8, np.float32):
        yield lambda dt=dt: P.test_counts_without_cap(7, dt)
    yield P.test_hollow_tetrahedron
    yield P.test_square
    yield lambda: P.test_regular_ngon(7)
    yield lambda: P.test_euler_characteristic_every_grade(12, np.int8, 22, 60.0)
    yield lambda: P.test_h0_deaths_are_mst_weights(22, np.float32)


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(tmp_path, name, old, new):
    import oracle
    src = oracle.source_text()
    assert src.count(old) >= 1, f"mutation site for '{name}' not found"
    lib = oracle.compile_variant(src.replace(old, new), str(tmp_path / "libmutant.so"))
    try:
        rc = subprocess.run([sys.executable, os.path.abspath(__file__), lib], cwd=ROOT,
                            capture_output=True, text=True, timeout=120).returncode
    except subprocess.TimeoutExpired:
        rc = "timeout"
    assert rc != 0, f"no pin caught the planted mistake '{name}'"


def test_unmutated_copy_passes(tmp_path):
    """Control: the same harness on an unedited copy catches nothing."""
    import oracle
    lib = oracle.compile_variant(oracle.source_text(), str(tmp_path / "libsame.so"))
    r = subprocess.run([sys.executable, os.path.abspath(__file__), lib], cwd=ROOT,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr


if __name__ == "__main__":
    sys.path[:0] = [ROOT, HERE]
    import oracle
    with oracle.using(sys.argv[1]):
        for pin in _pins():
            try:
                pin()
            except Exception as e:  # a pin caught the mistake
                print("caught:", type(e).__name__, e)
                sys.exit(1)
    sys.exit(0)
