"""Compile libdr.so (the CUDA library behind include/dr.h) for sm_103a.

Each translation unit is compiled in parallel with nvcc, then linked into an
in-tree shared library next to this file.  The CUDA runtime is linked as the
shared libcudart.so, so that the library and its host program (PyTorch, or a
C program) use one runtime: a second, static runtime does not know the host
program's pinned buffers and copies from them at a fraction of the link's
bandwidth the first time it sees each one.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libdr.so")
# the bounds-checked build (DR_CHECK_BOUNDS: every kernel index checked, an
# out-of-range one recorded in the plan's error word): a test build, never
# loaded by default
LIB_CHECKED = os.path.join(HERE, "libdr_checked.so")
SOURCES = ["dr_plan.cu", "dr_recon.cu", "dr_batch.cu", "dr_server.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# (diagnostic 177, "declared but never referenced": the array bounds some
# kernels compute are read only by the bounds-checked build's index macros)
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-diag-suppress", "177"]


def nvcc():
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found")
    return path


def _stale(lib=LIB):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(os.path.dirname(HERE), "include", "dr.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False, ptxas_info=False, checked=False):
    """Build libdr.so (checked=True: libdr_checked.so with DR_CHECK_BOUNDS)
    if any source is newer than it; returns its path."""
    lib = LIB_CHECKED if checked else LIB
    if not force and not _stale(lib):
        return lib
    cc = nvcc()
    tmp = tempfile.mkdtemp(prefix="drbuild")
    try:
        procs, objs = [], []
        for src in SOURCES:
            obj = os.path.join(tmp, src.replace(".cu", ".o"))
            cmd = [cc, *ARCH, *FLAGS, "-I", os.path.join(os.path.dirname(HERE), "include"),
                   "-c", os.path.join(CSRC, src), "-o", obj]
            if checked:
                cmd.append("-DDR_CHECK_BOUNDS")
            if ptxas_info:
                cmd += ["-Xptxas", "-v"]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE,
                                                stderr=subprocess.STDOUT, text=True)))
            objs.append(obj)
        failed = []
        for src, p in procs:
            out, _ = p.communicate()
            if p.returncode != 0:
                failed.append(f"--- {src}\n{out}")
            elif verbose or ptxas_info:
                print(out, file=sys.stderr)
        if failed:
            raise RuntimeError("nvcc failed:\n" + "\n".join(failed))
        tmp_lib = lib + f".tmp{os.getpid()}"
        cudalib = os.path.join(os.path.dirname(os.path.dirname(cc)), "lib64")
        subprocess.run([cc, *ARCH, "-shared", "-cudart", "shared", "-Xlinker", "-rpath",
                        "-Xlinker", cudalib, "-o", tmp_lib, *objs], check=True)
        os.replace(tmp_lib, lib)
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="-v" in sys.argv))
