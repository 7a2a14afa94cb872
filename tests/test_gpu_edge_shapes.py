"""Degenerate sizes through every kernel (rows, per-pixel, interval) against
the FP64 oracle: one pixel, two steps, one bin, slabs and tiles left partly
empty, bins entirely outside the swept depths, far more bins than steps.
Tolerance as in test_gpu_parity.py."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2201_13309_gb300 import dr  # noqa: E402
from tests.gen import synth  # noqa: E402

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-4
KERNELS = [("rows", {}), ("pixels", {"force_pixels": True}),
           ("intervals", {"force_intervals": True})]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()


def check(sc, kernel, kw, edge="leading"):
    plan = dr.Plan(sc.geom, sc.wires, sc.edges, edge=edge, **kw)
    assert plan.info()["kernel"] == kernel
    img = torch.from_numpy(np.ascontiguousarray(sc.images).view(np.int16)).cuda()
    out = plan.reconstruct(img)
    torch.cuda.synchronize()
    plan.check_device()
    got = out.cpu().numpy().astype(np.float64)
    ref = O.reconstruct(sc.geom, sc.wires, sc.images, sc.edges, edge)
    s = np.abs(np.diff(sc.images.astype(np.int64), axis=0)).sum(0)[None]
    err = np.abs(got - ref)
    assert not (err > FP32_TOL * s).any(), (err / np.maximum(s, 1)).max()
    assert np.all(got[np.broadcast_to(s == 0, got.shape)] == 0)
    return got


SHAPES = [  # rows, cols, K, bins (lo_um, hi_um, width_um)
    (1, 1, 2, (20.0, 20.0, 1.0)),      # one pixel, two steps, one bin
    (2, 3, 3, (10.0, 30.0, 10.0)),
    (3, 33, 5, (0.0, 60.0, 1.5)),      # a slab / tile with one column
    (2, 40, 3, (-100.0, 400.0, 1.0)),  # 501 bins for 2 intervals
    (4, 17, 9, (5.0, 50.0, 0.25)),
]


@pytest.mark.parametrize("kernel,kw", KERNELS, ids=[k for k, _ in KERNELS])
@pytest.mark.parametrize("shape", SHAPES, ids=[f"{s[0]}x{s[1]}x{s[2]}" for s in SHAPES])
def test_small_shapes(shape, kernel, kw):
    rows, cols, K, (lo, hi, w) = shape
    sc = synth.tiny_scan(rows * 1000 + cols * 10 + K, rows=rows, cols=cols, K=K, n_scat=3)
    sc.edges = synth.bin_edges(lo, hi, w)
    check(sc, kernel, kw)
    check(sc, kernel, kw, edge="trailing")


@pytest.mark.parametrize("kernel,kw", KERNELS, ids=[k for k, _ in KERNELS])
def test_bins_outside_swept_depths(kernel, kw):
    """Every bin lies beyond (or before) every pixel's depths: all zero."""
    sc = synth.tiny_scan(91, rows=4, cols=24, K=11)
    for lo, hi in ((900.0, 950.0), (-950.0, -900.0)):
        sc.edges = synth.bin_edges(lo, hi, 1.0)
        got = check(sc, kernel, kw)
        assert np.all(got == 0)


@pytest.mark.parametrize("kernel,kw", KERNELS, ids=[k for k, _ in KERNELS])
def test_empty_roi(kernel, kw):
    sc = synth.tiny_scan(92, rows=4, cols=8, K=5)
    for g in (dict(sc.geom, rows=0), dict(sc.geom, cols=0)):
        plan = dr.Plan(g, sc.wires, sc.edges, **kw)
        out = torch.empty((sc.B, g["rows"], g["cols"]), device="cuda")
        plan.reconstruct(torch.empty((5, g["rows"], g["cols"]), dtype=torch.int16,
                                     device="cuda"), out)
        torch.cuda.synchronize()
        plan.check_device()


def uneven_edges(seed, lo_um, hi_um):
    """Bin edges with widths drawn from 0.2 to 3 um: the kernels' edge
    searches start from a uniform-bin guess and must fall back to a binary
    search here."""
    rng = np.random.Generator(np.random.PCG64(seed))
    w = rng.uniform(0.2, 3.0, 400)
    e = lo_um + np.concatenate([[0.0], np.cumsum(w)])
    return e[e <= hi_um] * 1e-3


@pytest.mark.parametrize("kernel,kw", KERNELS, ids=[k for k, _ in KERNELS])
def test_uneven_bins(kernel, kw):
    sc = synth.tiny_scan(94, rows=6, cols=48, K=41)
    sc.edges = uneven_edges(94, -20.0, 70.0)
    assert np.ptp(np.diff(sc.edges)) > 2e-3
    check(sc, kernel, kw)


def test_uneven_bins_rows_and_pixels_bitwise():
    sc = synth.tiny_scan(95, rows=6, cols=64, K=41)
    sc.edges = uneven_edges(95, -20.0, 70.0)
    img = torch.from_numpy(np.ascontiguousarray(sc.images).view(np.int16)).cuda()
    a = dr.Plan(sc.geom, sc.wires, sc.edges).reconstruct(img)
    b = dr.Plan(sc.geom, sc.wires, sc.edges, force_pixels=True).reconstruct(img)
    torch.cuda.synchronize()
    assert torch.equal(a.view(torch.int32), b.view(torch.int32))


def test_uneven_bins_rotated():
    sc = synth.spot_scan(96, 4, 72, 33, 8, -60.0, 60.0, 1.0, rotate_deg=9.0,
                         depth_range=(-0.03, 0.03))
    sc.edges = uneven_edges(96, -70.0, 70.0)
    check(sc, "pixels", {})
