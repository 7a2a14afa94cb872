"""The oracle's pins catch plausible mistakes (CPU only).

Each mutant is a copy of oracle/oracle.c with one deliberate, plausible
error (a swapped edge, a flipped sign, a dropped term, a wrong index or
operand, an off-by-one).  It is compiled on the side and the pin suite
(tests/test_oracle_pins.py) is run against it: every mutant must fail at
least one pin.  The real oracle is never modified.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = {
    "edges swapped": ("int want_hi = edge == OR_LEADING ? lead_is_hi : !lead_is_hi;",
                      "int want_hi = edge == OR_LEADING ? !lead_is_hi : lead_is_hi;"),
    "difference sign flipped": ("dI[k] = J->edge == OR_LEADING ? a - b : b - a;",
                                "dI[k] = J->edge == OR_LEADING ? b - a : a - b;"),
    "normalisation dropped": ("(double)dI[k] * (b - a) / (hi - lo);",
                              "(double)dI[k] * (b - a);"),
    "bin shifted by one": ("if (b > a) out[(size_t)j * stride] +=",
                           "if (b > a) out[(size_t)(j + 1 < B ? j + 1 : j) * stride] +="),
    "atan for asin": ("double alpha = asin(f->radius / D);",
                      "double alpha = atan(f->radius / D);"),
    "projection index": ("  o[1] = v[1] - s * a[1];", "  o[1] = v[1] - s * a[0];"),
    "no projection of the pixel": ("  perp(qo, f->axis, qp);", "  memcpy(qp, qo, sizeof qp);"),
    "last interval dropped": ("  for (int k = 0; k + 1 < K; ++k) {\n    if (dI[k] == 0) continue;",
                              "  for (int k = 0; k + 2 < K; ++k) {\n    if (dI[k] == 0) continue;"),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name!r} not found exactly once"
    mut = tmp_path / "oracle_mutant.c"
    mut.write_text(src.replace(old, new))
    lib = tmp_path / "liboracle_mutant.so"
    subprocess.run(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-pthread", "-o", str(lib),
                    str(mut), "-lm"], check=True)
    env = dict(os.environ, DR_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        os.path.join(ROOT, "tests", "test_golden.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"no pin failed for mutant {name!r}:\n{r.stdout[-2000:]}"
