"""The reconstruction entry point that allocates nothing (GPU).

dr_reconstruct_rows_static serves callers that cannot call cudaMalloc (their
device memory belongs to another allocator, or their pipeline may not
allocate while running).  It keeps its geometry tables in a fixed device
array inside the library.  Its results must match the FP64 oracle within the
parity tolerance of the other GPU tests, and the plan-based entry point
(dr_plan + dr_reconstruct) within the same tolerance, call after call, even
though each call overwrites the array.  This file is collected last so a run
that stops at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2201_13309_gb300 import dr  # noqa: E402
from tests.gen import synth  # noqa: E402

pytestmark = pytest.mark.gpu
FP32_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()


def _dev(images):
    return torch.from_numpy(np.ascontiguousarray(images).view(np.int16)).cuda()


def _check_close(got, ref, images):
    s = np.abs(np.diff(images.astype(np.int64), axis=0)).sum(0)[None]
    err = np.abs(got.astype(np.float64) - ref.astype(np.float64))
    assert np.all(err <= FP32_TOL * s)
    assert np.all(got[np.broadcast_to(s == 0, got.shape)] == 0)


def _oracle(scan, r0=0, nrows=None):
    return O.reconstruct(scan.geom, scan.wires, scan.images, scan.edges, r0=r0, nrows=nrows)


def test_static_entry_matches_oracle_and_plan_entry_on_two_calls_in_a_row():
    a = synth.tiny_scan(21)                                  # 64x64, K=41, B=101
    b = synth.tiny_scan(22, rows=24, cols=203, K=77)         # one pixel per thread, ragged tile
    b.edges = synth.bin_edges(-20.0, 90.0, 0.5)
    b_back = synth.Scan(b.geom, b.wires[::-1].copy(), b.edges, b.images[::-1].copy())
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for scan in (a, b_back):
        plan = dr.Plan(scan.geom, scan.wires, scan.edges)
        img = _dev(scan.images)
        ref = plan.reconstruct(img)
        out = torch.full_like(ref, float("nan"))
        dr.reconstruct_rows_static(scan.geom, scan.wires, scan.edges, img, out, status)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        got = out.cpu().numpy()
        _check_close(got, _oracle(scan), scan.images)
        _check_close(got, ref.cpu().numpy(), scan.images)
    # the first scan again, with no status word, after the second one
    # overwrote the device tables
    out = torch.full((a.B, 64, 64), float("nan"), device="cuda")
    dr.reconstruct_rows_static(a.geom, a.wires, a.edges, _dev(a.images), out, status=None)
    torch.cuda.synchronize()
    _check_close(out.cpu().numpy(), _oracle(a), a.images)


def test_static_entry_tables_just_under_the_limit():
    """65480 rows of 6 pixels: 32 B of row constants per row bring the tables
    to within 256 bytes of the 2 MiB array."""
    H, W, K = 65480, 6, 41
    geom = synth.detector_geometry(H, W)
    geom["row_step"] = [0.0, 0.0, 0.003]
    geom["det_origin"] = [-(W - 1) / 2 * synth.PITCH_MM, synth.DET_Y_MM, -(H - 1) / 2 * 0.003]
    wires = synth.wire_path(K)
    edges = synth.bin_edges(-50.0, 50.0, 1.0)
    rng = np.random.Generator(np.random.PCG64(5))
    images = rng.integers(0, 4000, size=(K, H, W), dtype=np.uint16)
    scan = synth.Scan(geom, wires, edges, images)
    out = torch.full((scan.B, H, W), float("nan"), device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    dr.reconstruct_rows_static(geom, wires, edges, _dev(images), out, status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    got = out.cpu().numpy()
    for r0 in (0, H // 2, H - 40):
        _check_close(got[:, r0:r0 + 40], _oracle(scan, r0, 40), images[:, r0:r0 + 40])
    ref = dr.Plan(geom, wires, edges).reconstruct(_dev(images))
    _check_close(got, ref.cpu().numpy(), images)


def test_static_entry_refuses_stream_capture():
    """Inside a stream capture the call returns DR_ERR_UNSUPPORTED and queues
    nothing (the captured graph holds only the other work); the next call
    outside the capture runs normally."""
    a = synth.tiny_scan(23)
    img = _dev(a.images)
    out = torch.full((a.B, a.geom["rows"], a.geom["cols"]), float("nan"), device="cuda")
    x = torch.zeros(1, device="cuda")
    dr.reconstruct_rows_static(a.geom, a.wires, a.edges, img, out)  # device address looked up
    torch.cuda.synchronize()
    out.fill_(float("nan"))
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        x.add_(1.0)
        with pytest.raises(dr.DrError) as ei:
            dr.reconstruct_rows_static(a.geom, a.wires, a.edges, img, out)
    assert ei.value.status == 8
    assert "captured" in dr.lib().dr_last_error().decode()
    g.replay()
    torch.cuda.synchronize()
    assert float(x.item()) == 1.0
    assert bool(torch.isnan(out).all())
    dr.reconstruct_rows_static(a.geom, a.wires, a.edges, img, out)
    torch.cuda.synchronize()
    _check_close(out.cpu().numpy(), _oracle(a), a.images)


def _call_c(geom, wires, edges):
    """The C entry point itself, with null buffers (it must reject the
    request before it looks at them)."""
    w = np.ascontiguousarray(wires, dtype=np.float64)
    e = np.ascontiguousarray(edges, dtype=np.float64)
    g = dr.geometry_struct(geom)
    return dr.lib().dr_reconstruct_rows_static(
        ctypes.byref(g), w.ctypes.data_as(ctypes.c_void_p), w.shape[0],
        e.ctypes.data_as(ctypes.c_void_p), e.shape[0] - 1, None, None, None,
        ctypes.c_void_p(0))


def test_static_entry_rejects_what_does_not_fit():
    big = synth.detector_geometry(65500, 8)        # 65500 * 32 B of row tables > 2 MiB
    assert _call_c(big, synth.wire_path(41), synth.bin_edges(-50, 50, 1.0)) == 5
    assert "limit" in dr.lib().dr_last_error().decode()
    rot = synth.detector_geometry(8, 8, rotate_deg=10.0)
    assert _call_c(rot, synth.wire_path(5), synth.bin_edges(-5, 5, 1.0)) == 8
