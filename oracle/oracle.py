"""ctypes wrapper of the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of bench.py, never by the library.  It shares no
code with the CUDA path; both read the same geometry dicts produced by the
seeded generator.

Every function follows the steps listed in oracle.c (pixel centre, projection
onto the plane perpendicular to the wire axis, tangent-point depths, int64
differences, overlap apportioning).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

LEADING, TRAILING = 0, 1
_STATUS = {0: "ok", 1: "bad argument", 2: "bad geometry", 3: "out of memory"}


class OracleError(RuntimeError):
    pass


def build(force=False):
    """Compile oracle.c into liboracle.so with gcc (plain -O2, IEEE math)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-pthread",
                    "-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            i32 = ctypes.c_int
            lib.oracle_depths.argtypes = [P, i32, P, i32, i32, i32, i32, P]
            lib.oracle_depths.restype = i32
            lib.oracle_differences.argtypes = [P, i32, ctypes.c_longlong, P]
            lib.oracle_differences.restype = None
            lib.oracle_apportion.argtypes = [P, P, i32, ctypes.c_longlong, i32,
                                             P, i32, P]
            lib.oracle_apportion.restype = i32
            lib.oracle_reconstruct.argtypes = [P, i32, i32, P, i32, i32, P, P,
                                               i32, i32, i32, i32, P]
            lib.oracle_reconstruct.restype = i32
            _lib = lib
    return _lib


def _geom_array(geom):
    g = np.zeros(19, dtype=np.float64)
    g[0:3] = geom["beam_origin"]
    g[3:6] = geom["beam_dir"]
    g[6:9] = geom["det_origin"]
    g[9:12] = geom["row_step"]
    g[12:15] = geom["col_step"]
    g[15:18] = geom["wire_axis"]
    g[18] = geom["wire_radius"]
    return g


def _edge(edge):
    if edge in ("leading", LEADING):
        return LEADING
    if edge in ("trailing", TRAILING):
        return TRAILING
    raise ValueError(f"unknown edge {edge!r}")


def _check(st):
    if st != 0:
        raise OracleError(_STATUS.get(st, f"status {st}"))


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def depths(geom, wires, edge="leading", r0=0, nrows=None):
    """Depths [nrows, cols, K] (mm along the beam) of the chosen wire edge."""
    lib = _load()
    nrows = geom["rows"] - r0 if nrows is None else nrows
    wires = np.ascontiguousarray(wires, dtype=np.float64)
    K = wires.shape[0]
    out = np.empty((nrows, geom["cols"], K), dtype=np.float64)
    g = _geom_array(geom)
    _check(lib.oracle_depths(_ptr(g), geom["cols"], _ptr(wires), K, _edge(edge),
                             r0, nrows, _ptr(out)))
    return out


def differences(images):
    """int64 [K-1, ...] with dI_k = I_k - I_{k+1}."""
    lib = _load()
    im = np.ascontiguousarray(images, dtype=np.uint16)
    K = im.shape[0]
    P = int(np.prod(im.shape[1:])) if im.ndim > 1 else 1
    out = np.empty((max(K - 1, 0),) + im.shape[1:], dtype=np.int64)
    lib.oracle_differences(_ptr(im), K, P, _ptr(out))
    return out


def apportion(depth_seq, images, edges, edge="leading"):
    """Spread differences over bins for given depths.

    depth_seq: [P, K] float64; images: [K, P] uint16; edges: [B+1].
    Returns [B, P] float64.
    """
    lib = _load()
    d = np.ascontiguousarray(depth_seq, dtype=np.float64)
    im = np.ascontiguousarray(images, dtype=np.uint16)
    e = np.ascontiguousarray(edges, dtype=np.float64)
    P, K = d.shape
    B = e.shape[0] - 1
    out = np.empty((B, P), dtype=np.float64)
    _check(lib.oracle_apportion(_ptr(d), _ptr(im), K, P, _edge(edge), _ptr(e),
                                B, _ptr(out)))
    return out


def reconstruct(geom, wires, images, edges, edge="leading", r0=0, nrows=None,
                threads=None):
    """FP64 reconstruction of rows r0 .. r0+nrows-1: [B, nrows, cols].

    ``images`` is the whole ROI stack [K, rows, cols] (uint16).  edge "both"
    is the mean of the leading- and trailing-edge reconstructions.
    """
    if edge == "both":
        return 0.5 * (reconstruct(geom, wires, images, edges, "leading", r0, nrows, threads)
                      + reconstruct(geom, wires, images, edges, "trailing", r0, nrows, threads))
    lib = _load()
    H, W = geom["rows"], geom["cols"]
    nrows = H - r0 if nrows is None else nrows
    wires = np.ascontiguousarray(wires, dtype=np.float64)
    im = np.ascontiguousarray(images, dtype=np.uint16)
    e = np.ascontiguousarray(edges, dtype=np.float64)
    K = wires.shape[0]
    if im.shape != (K, H, W):
        raise ValueError(f"images shape {im.shape} != {(K, H, W)}")
    B = e.shape[0] - 1
    out = np.empty((B, nrows, W), dtype=np.float64)
    threads = threads or os.cpu_count() or 1
    g = _geom_array(geom)
    _check(lib.oracle_reconstruct(_ptr(g), H, W, _ptr(wires), K, _edge(edge),
                                  _ptr(im), _ptr(e), B, r0, nrows, threads,
                                  _ptr(out)))
    return out
