"""GPU parity of the interval kernel (depth sequences in any order) against
the FP64 oracle, through the C ABI.

The oracle adds every interval [min(d_k, d_{k+1}), max(d_k, d_{k+1})) by
itself (a zero-length interval into the bin holding it), which is the
definition the interval kernel follows; the running-sum kernels give the same
numbers for monotone sequences.  Tolerance as in test_gpu_parity.py: every
FP32 bin within 1e-4 x sum_k |dI_k| of its pixel.
"""
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


def to_dev(images):
    return torch.from_numpy(np.ascontiguousarray(images).view(np.int16)).cuda()


def assert_parity(got, ref, images, tol=FP32_TOL):
    got = np.asarray(got, dtype=np.float64)
    s = np.abs(np.diff(images.astype(np.int64), axis=0)).sum(0)[None]
    err = np.abs(got - ref)
    bad = err > tol * s
    assert not bad.any(), (
        f"{bad.sum()} bins off; worst err/sum|dI| = {(err / np.maximum(s, 1)).max():.3g}")
    assert np.all(got[np.broadcast_to(s == 0, got.shape)] == 0)


def run(sc, **kw):
    plan = dr.Plan(sc.geom, sc.wires, sc.edges, **kw)
    out = plan.reconstruct(to_dev(sc.images))
    torch.cuda.synchronize()
    plan.check_device()
    return plan, out


def mixed_scan(seed=5, rows=6, cols=24, K=41, roi=(1900, 1000)):
    """A wire that also climbs across the beam (3.5 um per 1 um step along
    it, with 0.4 um of seeded jitter): the depth of most steps runs against
    the wire's travel, some steps run with it."""
    rng = np.random.Generator(np.random.PCG64(seed))
    geom = synth.detector_geometry(rows, cols, roi_origin=roi, det_rows=2048, det_cols=2048)
    wires = synth.wire_path(K, dy=0.0035)
    wires[:, 1] += rng.normal(0.0, 0.0004, K)
    d = O.depths(geom, wires)
    lo, hi = d.min(), d.max()
    scat = synth.Scatterers(rng.uniform(lo, hi, 4), rng.uniform(500.0, 5000.0, 4))
    images = synth.poisson_u16(rng, synth.expected_counts(geom, wires, scat, background=30.0))
    edges = synth.bin_edges(np.floor(lo * 1e3) - 2, np.ceil(hi * 1e3) + 2, 0.5)
    return synth.Scan(geom, wires, edges, images), d


def test_mixed_direction_depths():
    sc, d = mixed_scan()
    steps = np.diff(d, axis=2)
    assert (steps < 0).any() and (steps > 0).any()
    plan, out = run(sc)
    assert plan.info()["kernel"] == "intervals"
    assert_parity(out.cpu().numpy(), O.reconstruct(sc.geom, sc.wires, sc.images, sc.edges),
                  sc.images)


def test_depth_against_wire_travel():
    """Every step of every pixel runs against the wire's travel (rejected by
    the running-sum kernels, taken by the interval kernel)."""
    sc = synth.tiny_scan(21, rows=4, cols=40, K=30, roi_origin=(1900, 1000), det_rows=2048,
                         det_cols=2048)
    sc.wires = synth.wire_path(30, dy=0.005)
    d = O.depths(sc.geom, sc.wires)
    assert (np.diff(d, axis=2) < 0).all()
    sc.edges = synth.bin_edges(np.floor(d.min() * 1e3) - 3, np.ceil(d.max() * 1e3) + 3, 1.0)
    plan, out = run(sc)
    assert plan.info()["kernel"] == "intervals"
    ref = O.reconstruct(sc.geom, sc.wires, sc.images, sc.edges)
    assert_parity(out.cpu().numpy(), ref, sc.images)


def test_repeated_wire_positions():
    """Two steps at the same centre: a zero-length interval, whose whole
    difference goes to the bin holding it."""
    sc = synth.tiny_scan(22, rows=8, cols=32, K=25)
    w = sc.wires.copy()
    w[7] = w[6]
    w[15] = w[14]
    sc.wires = w
    plan, out = run(sc)
    assert plan.info()["kernel"] == "intervals"
    assert_parity(out.cpu().numpy(), O.reconstruct(sc.geom, sc.wires, sc.images, sc.edges),
                  sc.images)


@pytest.mark.parametrize("edge", ["leading", "trailing", "both"])
def test_forced_on_monotone_scan_matches_running_sum(edge):
    """On a monotone scan the interval kernel and the rows kernel compute the
    same sum in a different order: both within the bar of the oracle and of
    each other; the bins of a pixel add up to its I_first - I_last."""
    sc = synth.tiny_scan(23, rows=12, cols=64, K=41)
    ref = O.reconstruct(sc.geom, sc.wires, sc.images, sc.edges, edge)
    plan, a = run(sc, edge=edge, force_intervals=True)
    assert plan.info()["kernel"] == "intervals"
    _, b = run(sc, edge=edge)
    a, b = a.cpu().numpy(), b.cpu().numpy()
    assert_parity(a, ref, sc.images)
    assert_parity(a, b, sc.images)
    if edge == "leading":
        d = O.depths(sc.geom, sc.wires)
        inside = (d.min(axis=2) > sc.edges[0]) & (d.max(axis=2) < sc.edges[-1])
        total = a.astype(np.float64).sum(0)
        want = sc.images[0].astype(np.float64) - sc.images[-1]
        s = np.abs(np.diff(sc.images.astype(np.int64), axis=0)).sum(0)
        assert np.all(np.abs(total - want)[inside] <= 1e-5 * np.maximum(s, 1)[inside])


@pytest.mark.parametrize("cols", [280, 283])
def test_forced_per_pixel_geometry(cols):
    """Rotated and tilted detector (constants per pixel), TMA-staged (280
    columns) and plain loads (283), reversed travel."""
    sc = synth.spot_scan(24, 3, cols, 37, 10, -60.0, 60.0, 0.7, rotate_deg=9.0, tilt_deg=3.0,
                         depth_range=(-0.03, 0.03))
    back = synth.Scan(sc.geom, sc.wires[::-1].copy(), sc.edges, sc.images[::-1].copy())
    for s in (sc, back):
        plan, out = run(s, force_intervals=True)
        info = plan.info()
        assert (info["kernel"], info["tile_cols"]) == ("intervals", 32)
        assert_parity(out.cpu().numpy(), O.reconstruct(s.geom, s.wires, s.images, s.edges),
                      s.images)


def test_bins_in_several_windows():
    """More bins than one shared-memory window holds."""
    sc = synth.tiny_scan(25, rows=2, cols=16, K=101)
    sc.edges = synth.bin_edges(-150.0, 150.0, 0.05)
    plan, out = run(sc, force_intervals=True)
    info = plan.info()
    assert info["bin_groups"] < info["B"]  # bins per window
    assert_parity(out.cpu().numpy(), O.reconstruct(sc.geom, sc.wires, sc.images, sc.edges),
                  sc.images)


def test_back_and_forth_in_one_plan():
    """A path that turns back along the beam, as one interval plan (the
    running-sum kernels split it into runs)."""
    a = synth.wire_path(24)
    b = synth.wire_path(11, z0=a[-1, 2], dz=-0.001)[1:]
    c = synth.wire_path(15, z0=b[-1, 2], dz=0.001)[1:]
    wires = np.concatenate([a, b, c])
    geom = synth.detector_geometry(12, 64, roi_origin=(26, 0), det_rows=64, det_cols=64)
    rng = np.random.Generator(np.random.PCG64(26))
    images = synth.poisson_u16(
        rng, synth.expected_counts(geom, wires, synth.tiny_scatterers(rng, 4)))
    sc = synth.Scan(geom, wires, synth.bin_edges(-40, 60, 1.0), images)
    plan, out = run(sc, force_intervals=True)
    assert plan.info()["parts"] == 1
    assert_parity(out.cpu().numpy(), O.reconstruct(geom, wires, images, sc.edges), images)


def test_variants_streamed_fp64_bf16_deterministic():
    sc, _ = mixed_scan(seed=6, rows=10, cols=40)
    ref = O.reconstruct(sc.geom, sc.wires, sc.images, sc.edges)
    plan, out = run(sc)
    assert plan.info()["kernel"] == "intervals"
    _, again = run(sc)
    assert torch.equal(out.view(torch.int32), again.view(torch.int32))
    # streamed slabs of rows: bitwise the device-resident result
    h_img = torch.from_numpy(sc.images.view(np.int16)).pin_memory()
    h_out = torch.empty(tuple(out.shape)).pin_memory()
    ws = torch.empty(4 << 20, dtype=torch.uint8, device="cuda")
    plan.reconstruct_streamed(h_img, h_out, ws, slab_rows=3)
    torch.cuda.synchronize()
    assert torch.equal(h_out.view(torch.int32), out.cpu().view(torch.int32))
    # FP64 geometry
    p64, o64 = run(sc, geom_precision="fp64")
    assert p64.info()["kernel"] == "intervals"
    assert_parity(o64.cpu().numpy(), ref, sc.images, tol=1e-6)
    # BF16 output: 2^-8 of the magnitude plus the FP32 bar
    _, ob = run(sc, out_dtype="bf16")
    got = ob.float().cpu().numpy().astype(np.float64)
    s = np.abs(np.diff(sc.images.astype(np.int64), axis=0)).sum(0)[None]
    assert np.all(np.abs(got - ref) <= FP32_TOL * s + 2.0 ** -8 * np.abs(ref))


def test_both_edges_mixed_depths():
    sc, _ = mixed_scan(seed=7)
    plan, out = run(sc, edge="both")
    info = plan.info()
    assert (info["kernel"], info["parts"]) == ("intervals", 2)
    assert_parity(out.cpu().numpy(),
                  O.reconstruct(sc.geom, sc.wires, sc.images, sc.edges, "both"), sc.images)


def test_per_pixel_geometry_in_several_windows():
    """Rotated detector (depths per pixel) with more bins than one window
    holds, a ragged last tile of 32 pixels (70 columns), reversed travel."""
    sc = synth.spot_scan(27, 3, 70, 101, 6, -60.0, 60.0, 0.7, rotate_deg=12.0,
                         depth_range=(-0.03, 0.03))
    sc.edges = synth.bin_edges(-150.0, 150.0, 0.05)
    back = synth.Scan(sc.geom, sc.wires[::-1].copy(), sc.edges, sc.images[::-1].copy())
    for s in (sc, back):
        plan, out = run(s, force_intervals=True)
        info = plan.info()
        assert info["kernel"] == "intervals" and info["bin_groups"] < info["B"]
        assert_parity(out.cpu().numpy(), O.reconstruct(s.geom, s.wires, s.images, s.edges),
                      s.images)


@pytest.mark.parametrize("rotate,edge,backward", [(0.0, "leading", False),
                                                   (9.0, "leading", False),
                                                   (9.0, "trailing", False),
                                                   (0.0, "leading", True)])
def test_steps_too_fine_for_fp32_positions(rotate, edge, backward):
    """A step of 1 pm is below what the FP32 positions' grid resolves: the
    interval kernel apportions that interval with its depths in FP64.  A bin
    edge is put inside the short interval of row 0, so its difference is
    split between two bins; FP32 plan, within the FP32 bar of the oracle;
    trailing edge and a reversed scan included."""
    sc = synth.tiny_scan(28, rows=6, cols=40, K=41, rotate_deg=rotate)
    w = sc.wires.copy()
    w[20:, 2] -= 0.001 - 1e-9
    sc.wires = w
    if backward:
        sc = synth.Scan(sc.geom, sc.wires[::-1].copy(), sc.edges, sc.images[::-1].copy())
    d = O.depths(sc.geom, sc.wires, edge)
    k = 20 if backward else 19  # the short interval joins steps k and k + 1
    mid = 0.5 * (d[0, 0, k] + d[0, 0, k + 1])
    edges = synth.bin_edges(-50.0, 90.0, 1.0)
    j = int(np.searchsorted(edges, mid))
    sc.edges = edges + (mid - edges[j])
    plan, out = run(sc, edge=edge)
    info = plan.info()
    assert (info["kernel"], info["geom_precision"]) == ("intervals", 0)  # FP32
    assert_parity(out.cpu().numpy(),
                  O.reconstruct(sc.geom, sc.wires, sc.images, sc.edges, edge), sc.images)
