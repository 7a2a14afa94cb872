"""The oracle's pins catch plausible mistakes (CPU only).

Each mutant is a copy of the oracle (oracle/oracle.c or oracle/oracle.py)
with one deliberate, plausible error (a swapped edge, a flipped sign, a
dropped term, a wrong index or operand, an off-by-one, a wrong weight).  The
oracle and the pin tests are copied into a scratch tree, the mutation is
applied there, and the pin suite (tests/test_oracle_pins.py with the golden
fixture test) runs against the copy: every mutant must fail at least one
pin.  The real oracle is never modified.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C, PY = "oracle.c", "oracle.py"
MUTANTS = {
    "edges swapped": (C, "int want_hi = edge == OR_LEADING ? lead_is_hi : !lead_is_hi;",
                      "int want_hi = edge == OR_LEADING ? !lead_is_hi : lead_is_hi;"),
    "difference sign flipped": (C, "dI[k] = J->edge == OR_LEADING ? a - b : b - a;",
                                "dI[k] = J->edge == OR_LEADING ? b - a : a - b;"),
    "trailing-edge sign flipped": (C, "dI[k] = J->edge == OR_LEADING ? a - b : b - a;",
                                   "dI[k] = J->edge == OR_LEADING ? a - b : a - b;"),
    "normalisation dropped": (C, "(double)dI[k] * (b - a) / (hi - lo);",
                              "(double)dI[k] * (b - a);"),
    "bin shifted by one": (C, "if (b > a) out[(size_t)j * stride] +=",
                           "if (b > a) out[(size_t)(j + 1 < B ? j + 1 : j) * stride] +="),
    "atan for asin": (C, "double alpha = asin(f->radius / D);",
                      "double alpha = atan(f->radius / D);"),
    "projection index": (C, "  o[1] = v[1] - s * a[1];", "  o[1] = v[1] - s * a[0];"),
    "no projection of the pixel": (C, "  perp(qo, f->axis, qp);", "  memcpy(qp, qo, sizeof qp);"),
    "last interval dropped": (C, "  for (int k = 0; k + 1 < K; ++k) {\n    if (dI[k] == 0) continue;",
                              "  for (int k = 0; k + 2 < K; ++k) {\n    if (dI[k] == 0) continue;"),
    "interval ends not ordered": (C, "double lo = d[k] < d[k + 1] ? d[k] : d[k + 1];",
                                  "double lo = d[k];"),
    "zero-length interval dropped": (C, "if (j >= 0) out[(size_t)j * stride] += (double)dI[k];",
                                     "if (j >= 0 && 0) out[(size_t)j * stride] += (double)dI[k];"),
    "edge counted in the lower bin": (C, "if (e[mid] <= x) lo = mid; else hi = mid;",
                                      "if (e[mid] < x) lo = mid; else hi = mid;"),
    "overlap over the bin width": (C, "(double)dI[k] * (b - a) / (hi - lo);",
                                   "(double)dI[k] * (b - a) / (e[j + 1] - e[j]);"),
    "overlap end not clipped": (C, "double b = hi < e[j + 1] ? hi : e[j + 1];",
                                "double b = hi < e[j + 1] ? e[j + 1] : hi;"),
    "beam direction not normalised": (C, "double b[3] = {g[3] / nb, g[4] / nb, g[5] / nb};",
                                      "double b[3] = {g[3], g[4], g[5]};"),
    "wire axis not normalised": (C, "f->axis[i] = g[15 + i] / na;", "f->axis[i] = g[15 + i];"),
    "travel from the first step": (C, "double move[3] = {wires[3 * (K - 1)] - wires[0], "
                                      "wires[3 * (K - 1) + 1] - wires[1],\n"
                                      "                    wires[3 * (K - 1) + 2] - wires[2]};",
                                   "double move[3] = {wires[3] - wires[0], wires[4] - wires[1],\n"
                                   "                    wires[5] - wires[2]};"),
    "depth over |b'| instead of b'.b'": (C, "d[s] = dot3(x, f->bproj) / f->bb;",
                                         "d[s] = dot3(x, f->bproj) / sqrt(f->bb);"),
    "rows and columns swapped": (C, "q[i] = g[6 + i] + r * g[9 + i] + c * g[12 + i];",
                                 "q[i] = g[6 + i] + c * g[9 + i] + r * g[12 + i];"),
    "wire not taken relative to the beam origin": (
        C, "double co[3] = {c[0] - f->origin[0], c[1] - f->origin[1], c[2] - f->origin[2]};",
        "double co[3] = {c[0], c[1], c[2]};"),
    "lower depth taken from one tangent": (C, "*lo = d[0] < d[1] ? d[0] : d[1];", "*lo = d[0];"),
    "row offset ignored (reconstruction)": (C, "int r = J->r0 + rr;", "int r = rr;"),
    "row offset ignored (depths)": (C, "st = pixel_depths(geom, &f, wires, K, edge, r0 + r, c,",
                                    "st = pixel_depths(geom, &f, wires, K, edge, r, c,"),
    "no refusal of a beam met before the wire": (
        C, "if (!(t > sqrt(D * D - f->radius * f->radius))) return OR_BAD_GEOMETRY;", ";"),
    "no refusal of a path without travel": (
        C, "if (along == 0.0) return OR_BAD_GEOMETRY; /* no travel along the beam */", ";"),
    "beam not projected onto the plane": (C, "perp(b, f->axis, f->bproj);",
                                          "memcpy(f->bproj, b, sizeof b);"),
    "one tangent taken twice": (C, "double th = s == 0 ? alpha : -alpha;", "double th = alpha;"),
    "tangent parameter sign": (C, "double t = -dot3(qxb, f->axis) / den;",
                               "double t = dot3(qxb, f->axis) / den;"),
    "travel sign inverted": (C, "int lead_is_hi = f->travel > 0;", "int lead_is_hi = f->travel < 0;"),
    "overlap start not clipped": (C, "double a = lo > e[j] ? lo : e[j];", "double a = e[j];"),
    "both edges summed, not averaged": (PY, "return 0.5 * (reconstruct(",
                                        "return 1.0 * (reconstruct("),
    "both edges: trailing twice": (PY, '+ reconstruct(geom, wires, images, edges, "trailing"',
                                   '+ reconstruct(geom, wires, images, edges, "leading"'),
}


def _copy_tree(dst):
    ignore = shutil.ignore_patterns("__pycache__", "*.so", "*.so.tmp*")
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(dst, "oracle"), ignore=ignore)
    shutil.copytree(os.path.join(ROOT, "tests"), os.path.join(dst, "tests"), ignore=ignore)


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    fname, old, new = MUTANTS[name]
    _copy_tree(str(tmp_path))
    path = tmp_path / "oracle" / fname
    src = path.read_text()
    assert src.count(old) == 1, f"mutation site for {name!r} not found exactly once"
    path.write_text(src.replace(old, new))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join("tests", "test_oracle_pins.py"),
                        os.path.join("tests", "test_golden.py")],
                       cwd=str(tmp_path), capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"no pin failed for mutant {name!r}:\n{r.stdout[-2000:]}"
    assert " failed" in r.stdout, "the pin run did not get as far as the pins:\n" + r.stdout[-2000:]


def test_unmutated_copy_passes(tmp_path):
    """The scratch-tree copy itself passes every pin (so a mutant's failure is
    the mutation's doing, not the copy's)."""
    _copy_tree(str(tmp_path))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join("tests", "test_oracle_pins.py"),
                        os.path.join("tests", "test_golden.py")],
                       cwd=str(tmp_path), capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
