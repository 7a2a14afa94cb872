"""The C ABI from a plain C program: tests/c/abi_consumer.c is compiled with
gcc against include/dr.h and the in-tree libdr.so and run; it plans,
reconstructs and checks conservation by itself."""
import os
import shutil
import subprocess

import pytest

torch = pytest.importorskip("torch")

from paper_2201_13309_gb300 import _build  # noqa: E402

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_plain_c_consumer(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lib = _build.build()
    cuda = os.path.dirname(os.path.dirname(_build.nvcc()))
    exe = tmp_path / "abi_consumer"
    subprocess.run([cc, "-O2", "-std=c99", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(cuda, "include"),
                    os.path.join(ROOT, "tests", "c", "abi_consumer.c"), "-o", str(exe),
                    "-L", os.path.dirname(lib), "-ldr", "-L", os.path.join(cuda, "lib64"),
                    "-lcudart", "-lm", f"-Wl,-rpath,{os.path.dirname(lib)}",
                    f"-Wl,-rpath,{os.path.join(cuda, 'lib64')}"], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "abi consumer ok" in r.stdout
