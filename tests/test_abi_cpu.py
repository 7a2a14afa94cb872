"""The C ABI library loads, exports every declared symbol, and validates its
inputs on the host (no GPU needed: every case fails before any CUDA call)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2201_13309_gb300 import _build, dr
from tests.gen import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return dr.lib()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "dr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dr_[a-z0-9_]+)\s*\(", text)))


def test_header_declarations_match_binding():
    assert set(declared_symbols()) == set(dr.EXPORTS)


def test_library_exports_every_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert dr.version() == "1.0.0"
    assert lib.dr_status_string(3).decode().startswith("depth not monotone")


def _plan_status(geom, wires, edges, edge="leading"):
    L = dr.lib()
    g = dr.geometry_struct(geom, edge)
    w = np.ascontiguousarray(wires, dtype=np.float64)
    e = np.ascontiguousarray(edges, dtype=np.float64)
    h = ctypes.c_void_p()
    st = L.dr_plan(ctypes.byref(g), w.ctypes.data_as(ctypes.c_void_p), w.shape[0],
                   e.ctypes.data_as(ctypes.c_void_p), e.shape[0] - 1, None,
                   ctypes.byref(h))
    assert not h.value
    return st, L.dr_last_error().decode()


def test_plan_rejects_bad_inputs(lib):
    g = synth.detector_geometry(8, 8)
    w = synth.wire_path(5)
    e = synth.bin_edges(-10, 10, 1.0)
    assert _plan_status(g, w[:1], e)[0] == 1                     # K < 2
    assert _plan_status(g, w, e[:1])[0] == 1                     # B < 1
    bad = e.copy()
    bad[3] = bad[2]
    assert _plan_status(g, w, bad)[0] == 1                       # not increasing
    g2 = dict(g, beam_dir=[1.0, 0.0, 0.0])
    assert _plan_status(g2, w, e)[0] == 2                        # beam along wire
    still = np.repeat(w[:1], 5, axis=0)
    assert _plan_status(g, still, e)[0] == 2                     # no travel
    low = w.copy()
    low[:, 1] = 0.01
    assert _plan_status(g, low, e)[0] == 2                       # wire hits beam
    far = w.copy()
    far[:, 1] = 600.0
    assert _plan_status(g, far, e)[0] == 2                       # wire past detector
    back = np.concatenate([w, w[::-1][1:]])
    assert _plan_status(g, back, e)[0] == 2                      # ends where it began
    assert _plan_status(g, back, e, edge="both")[0] == 2         # both edges, same
    g3 = dict(g, rows=-1)
    assert _plan_status(g3, w, e)[0] == 1
    fine = synth.wire_path(5, dz=1e-10)                          # 0.1 pm steps
    st, msg = _plan_status(g, fine, e)
    assert st == 8 and "too small" in msg                        # FP32 grid limit
    # (on a GPU the interval kernel takes such a scan, its short intervals
    # with FP64 depths: test_gpu_intervals.py)
    # Repeated positions and depths running against the wire's travel are
    # valid plans (the interval kernel): they get past validation to the
    # device allocation, tested in test_gpu_intervals.py.


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(dr, "LIB_PATH", str(tmp_path / "libdr.so"))
    monkeypatch.setattr(dr, "_lib", None)
    with pytest.raises(ImportError):
        dr.lib()


def test_static_entry_binding_checks_buffers_before_any_call(monkeypatch):
    """The no-allocation entry point cannot see buffer sizes; the binding
    refuses a wrong shape, type or device before it reaches the library."""
    import torch

    def no_call():
        raise AssertionError("the library was called")

    monkeypatch.setattr(dr, "lib", no_call)
    sc = synth.tiny_scan(3, rows=4, cols=8, K=5)
    K, H, W, B = sc.K, 4, 8, sc.B
    img = torch.zeros((K, H, W), dtype=torch.int16)
    good_out = torch.zeros((B, H, W), dtype=torch.float32)
    cases = [
        (sc.wires.reshape(-1), sc.edges, img, good_out),              # wires not [K, 3]
        (sc.wires, sc.edges[:, None], img, good_out),                 # edges not 1-D
        (sc.wires, sc.edges, img, torch.zeros((B, H, W - 1))),        # out too small
        (sc.wires, sc.edges, img, torch.zeros((B, H, W), dtype=torch.float64)),
        (sc.wires, sc.edges, torch.zeros((K, H, W), dtype=torch.int32), good_out),
        (sc.wires, sc.edges, img[:, :, ::2], torch.zeros((B, H, 4))),  # wrong shape
        (sc.wires, sc.edges, None, good_out),
        (sc.wires, sc.edges, img, good_out),                          # host tensors
    ]
    for wires, edges, images, out in cases:
        with pytest.raises(ValueError):
            dr.reconstruct_rows_static(sc.geom, wires, edges, images, out)
    with pytest.raises(ValueError):
        dr.reconstruct_rows_static(sc.geom, sc.wires, sc.edges, img, good_out,
                                   status=torch.zeros(2, dtype=torch.int32))


def _unbuilt_plan(K, rows, cols, B, out_dtype="f32"):
    """A Plan object with the attributes its methods check, but no library
    plan behind it (dr_plan needs a GPU)."""
    p = object.__new__(dr.Plan)
    p._h = ctypes.c_void_p()
    p.K, p.rows, p.cols, p.B, p.out_dtype = K, rows, cols, B, out_dtype
    return p


def test_binding_checks_buffers_before_any_call(monkeypatch):
    """Every entry point that hands the library a buffer by address checks
    its shape, element type, contiguity and memory (device or host) first:
    a wrong one raises ValueError and the library is never called."""
    import torch

    def no_call():
        raise AssertionError("the library was called")

    monkeypatch.setattr(dr, "lib", no_call)
    K, H, W, B = 5, 4, 8, 11
    p = _unbuilt_plan(K, H, W, B)
    img = torch.zeros((K, H, W), dtype=torch.int16)
    out = torch.zeros((B, H, W), dtype=torch.float32)
    bad = [
        lambda: p.reconstruct(img, out),                                    # host tensors
        lambda: p.reconstruct(torch.zeros((K, H, W + 1), dtype=torch.int16), out),
        lambda: p.reconstruct(img.float(), out),
        lambda: p.reconstruct(img, out.double()),
        lambda: p.reconstruct(img, out.transpose(1, 2).contiguous().transpose(1, 2)),
        lambda: p.reconstruct_host(img, out.half(), img, out),              # host output type
        lambda: p.reconstruct_host(img, torch.zeros((B, H, W - 1)), img, out),
        lambda: p.reconstruct_host(img, out, img, out),                     # "device" on host
        lambda: p.reconstruct_streamed(img, out.half(), torch.zeros(64, dtype=torch.uint8)),
        lambda: p.reconstruct_streamed(img[:, :, ::2], out, torch.zeros(64, dtype=torch.uint8)),
        lambda: p.reconstruct_streamed(img, out, torch.zeros(64, dtype=torch.uint8)),
        lambda: p.reconstruct_selected(torch.zeros((K, H, W - 1), dtype=torch.int16),
                                       torch.zeros(3, dtype=torch.int32), 3),
        lambda: dr.image_differences(img.float()),
        lambda: dr.image_differences(img),
        lambda: dr.pixel_activity(img[:, :, ::2]),
        lambda: dr.select_pixels(torch.zeros(16, dtype=torch.float64), 0.5),
        lambda: dr.select_pixels(torch.zeros(16), 0.5),
    ]
    for i, f in enumerate(bad):
        with pytest.raises(ValueError):
            f()
    srv = object.__new__(dr.Server)
    srv._h, srv._pinned = ctypes.c_void_p(), {}
    sc = synth.tiny_scan(3, rows=H, cols=W, K=K)
    for h in (torch.zeros((K - 1, H, W), dtype=torch.int16),
              torch.zeros((K, H, W), dtype=torch.float32),
              torch.zeros((K, W, H), dtype=torch.int16).transpose(1, 2)):
        with pytest.raises(ValueError):
            srv.submit(sc.geom, sc.wires, sc.edges, h)
    with pytest.raises(ValueError):
        srv.submit(sc.geom, sc.wires.reshape(-1), sc.edges, torch.zeros((K, H, W), dtype=torch.int16))
