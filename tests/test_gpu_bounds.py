"""The bounds-checked build (GPU): libdr_checked.so, compiled with
DR_CHECK_BOUNDS, checks every shared-memory and global index of the
reconstruction kernels and records the first out-of-range one in the plan's
error word instead of touching memory outside its array.  Edge shapes
(tests/bounds_shapes.py) run through every kernel in a process of its own
that loads the checked build; every error word must stay clear and every
result match the oracle."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_runs_the_edge_shapes_clean():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_13309_gb300 import _build

    lib = _build.build(checked=True)
    env = dict(os.environ, DR_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "bounds_shapes.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "clean" in r.stdout
