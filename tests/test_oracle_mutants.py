"""Planted mistakes in a copy of the oracle must be caught by the pins.

Each mutant is one plausible slip (a dropped term, a wrong sign or index, a
flipped tie rule) applied textually to a temporary copy of oracle/oracle.c.
The copy is compiled on the CPU and the pin tests are run against it in a
subprocess (ORACLE_LIB points the oracle front end at the mutant build); they
must fail.  The real oracle source is never modified.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = {
    "E_drops_extension": ("max2(H[i * w + j - 1] + p->GO, E[i * w + j - 1] + p->GE)",
                          "max2(H[i * w + j - 1] + p->GO, E[i * w + j - 1])"),
    "F_extends_with_open": ("max2(H[(i - 1) * w + j] + p->GO, F[(i - 1) * w + j] + p->GE)",
                            "max2(H[(i - 1) * w + j] + p->GO, F[(i - 1) * w + j] + p->GO)"),
    "mismatch_sign": ("(T[i - 1] == R[j - 1] ? p->a : p->b);\n            int32_t h",
                      "(T[i - 1] == R[j - 1] ? p->a : -p->b);\n            int32_t h"),
    "diagonal_wrong_cell": ("int32_t g = H[(i - 1) * w + j - 1] + (T",
                            "int32_t g = H[(i - 1) * w + j] + (T"),
    "glocal_boundary_off_by_one": ("p->GO + (j - 1) * p->GE", "p->GO + j * p->GE"),
    "no_local_floor": ("if (p->mode == OR_LOCAL) h = max2(h, 0);", ""),
    "best_tie_takes_last": ("if (H[i * w + j] > best)", "if (H[i * w + j] >= best)"),
    "second_exclusion_off_by_one": ("if (d < n) continue;", "if (d <= n) continue;"),
    "traceback_prefers_I_over_D": ("else if (h == F[i * w + j]) st = ST_F;\n            else st = ST_E;",
                                   "else if (h == E[i * w + j]) st = ST_E;\n            else st = ST_F;"),
    "D_ties_extend": ("F[(i - 1) * w + j] + p->GE > H[(i - 1) * w + j] + p->GO",
                      "F[(i - 1) * w + j] + p->GE >= H[(i - 1) * w + j] + p->GO"),
    "I_ties_extend": ("E[i * w + j - 1] + p->GE > H[i * w + j - 1] + p->GO",
                      "E[i * w + j - 1] + p->GE >= H[i * w + j - 1] + p->GO"),
    "soft_clip_dropped": ("push_op(ops, &n_ops, OP_S, n - res->read_end);", ""),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) >= 1, f"mutation anchor for {name} not found"
    mutated = text.replace(old, new, 1)
    src = tmp_path / "oracle_mutant.c"
    src.write_text(mutated)
    lib = tmp_path / "liboracle_mutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", str(src),
                           "-o", str(lib)])
    env = dict(os.environ, ORACLE_LIB=str(lib))
    proc = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                           os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                           os.path.join(ROOT, "tests", "test_oracle_bruteforce.py")],
                          env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert proc.returncode != 0, f"mutant {name} passed every pin:\n{proc.stdout[-2000:]}"
