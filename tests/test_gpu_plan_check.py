"""The plan's check of every (pixel, step) (GPU).

For FP32 geometry the running-sum kernels need every depth sequence to
increase, with steps the fixed-point grid takes.  dr_plan computes every
(row or pixel, step) depth exactly as the kernels will and compares it with
the FP64 solution; these tests hold its findings against the FP64 oracle
evaluated at every pixel, and check that a geometry whose depth steps change
sign inside the ROI goes to the interval kernel and still matches the
oracle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2201_13309_gb300 import dr  # noqa: E402
from tests.gen import synth  # noqa: E402
from tests.test_gpu_parity import assert_parity, ref_of, run  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()


@pytest.mark.parametrize("rotate,tilt", [(10.0, 0.0), (23.0, 6.0)])
def test_plan_reports_every_pixels_steps(rotate, tilt):
    """Smallest and largest step and the largest depth error, as the plan
    reports them, against the oracle's depths of every pixel."""
    sc = synth.spot_scan(8, 37, 70, 29, 6, -60, 60, 1.0, roi_origin=(300, 900),
                         det_rows=2048, det_cols=2048, rotate_deg=rotate, tilt_deg=tilt)
    plan = dr.Plan(sc.geom, sc.wires, sc.edges)
    info = plan.info()
    assert info["kernel"] == "pixels"
    assert info["checked_groups"] == 37 * 70
    unit = 2.0 ** -info["fixed_shift"]
    d = O.depths(sc.geom, sc.wires)                 # [rows, cols, K], every pixel
    steps = np.diff(d, axis=2)
    assert abs(info["min_step"] - steps.min()) < 8 * unit
    assert abs(info["max_step"] - steps.max()) < 8 * unit
    gpu = plan.depths().cpu().numpy()
    err = np.abs(gpu - d).max()
    assert 0 <= info["depth_err"] < 4 * unit
    assert abs(err - info["depth_err"]) < 1.5 * unit + 1e-12
    assert_parity(plan.reconstruct(torch.from_numpy(sc.images.view(np.int16)).cuda())
                  .cpu().numpy(), ref_of(sc), sc.images)


def test_polynomial_form_on_the_beamline_geometry():
    """The beamline scan takes the polynomial form of the remainder; its
    depths stay within the FP32 bar of the oracle, for the rows and the
    per-pixel plans."""
    sc = synth.tiny_scan(5)
    for kw in ({}, {"force_pixels": True}):
        plan = dr.Plan(sc.geom, sc.wires, sc.edges, **kw)
        info = plan.info()
        assert info["depth_form"] == 2 and info["one_step_per_bin"] == 1
        unit = 2.0 ** -info["fixed_shift"]
        err = np.abs(plan.depths().cpu().numpy() - O.depths(sc.geom, sc.wires)).max()
        assert err < 4 * unit and info["depth_err"] < 4 * unit


def _step_sign_change_scan(band_row):
    """A rotated ROI of 40 x 24 pixels (the plan's host pre-check samples
    rows 0, 16, 32, 39) and a wire that, at one step, also climbs toward the
    detector: that step's depth change is positive for pixels below a line
    through row band_row + 0.5 and negative above it."""
    H, W, K, k_star = 40, 24, 12, 6
    geom = synth.detector_geometry(H, W, roi_origin=(1700, 1000), det_rows=2048,
                                   det_cols=2048, rotate_deg=3.0)
    wires = synth.wire_path(K)
    base = O.depths(geom, wires)
    z_rows = np.asarray(geom["det_origin"])[2] + np.arange(H) * geom["row_step"][2]
    z_star = 0.5 * (z_rows[band_row] + z_rows[band_row + 1])
    # depth step ~ dz (D + y0) / D - deta (Z - z) / D: zero at Z = z_star
    D = synth.DET_Y_MM - synth.WIRE_Y_MM
    deta = 1e-3 * (D + synth.WIRE_Y_MM) / (z_star - wires[k_star, 2])
    wires[k_star:, 1] += deta
    d = O.depths(geom, wires)
    st = d[:, :, k_star] - d[:, :, k_star - 1]
    assert (st[:band_row - 1] > 0).all() and (st[band_row + 2:] < 0).all(), base.shape
    rng = np.random.Generator(np.random.PCG64(12))
    scat = synth.Scatterers(rng.uniform(d.min(), d.max(), 4), rng.uniform(500.0, 5000.0, 4))
    images = synth.poisson_u16(rng, synth.expected_counts(geom, wires, scat, background=25.0))
    return synth.Scan(geom, wires, synth.bin_edges(-40.0, 60.0, 1.0), images)


@pytest.mark.parametrize("band_row", [5, 23, 36])
def test_step_sign_change_between_sampled_rows_takes_interval_kernel(band_row):
    """The per-pixel plan's device check finds the pixels whose depth falls
    at one step and sends the scan to the interval kernel, even when the
    per-pixel kernel is asked for; the result matches the oracle."""
    sc = _step_sign_change_scan(band_row)
    for kw in ({}, {"force_pixels": True}):
        plan, out = run(sc, **kw)
        assert plan.info()["kernel"] == "intervals"
        assert_parity(out.cpu().numpy(), ref_of(sc), sc.images)


@pytest.mark.parametrize("form", ["exact", "series", "poly"])
def test_each_depth_form_against_the_oracle(form):
    """Every form of the FP32 remainder (exact, series of dL, per-pixel
    cubic in the wire position), asked for explicitly: depths within the
    FP32 bar of the oracle, the plan's own error figure consistent with
    them, and the reconstruction within tolerance; rows and per-pixel plans."""
    rot = synth.spot_scan(9, 20, 64, 41, 6, -60, 60, 1.0, roi_origin=(1000, 300),
                          det_rows=2048, det_cols=2048, rotate_deg=12.0, tilt_deg=3.0,
                          depth_range=(-0.03, 0.03))
    row = synth.spot_scan(10, 30, 48, 45, 6, -60, 60, 1.0, roi_origin=(1800, 0),
                          det_rows=2048, det_cols=2048, depth_range=(-0.03, 0.03))
    want = {"exact": 0, "series": 1, "poly": 2}[form]
    for sc, kernel in ((rot, "pixels"), (row, "rows")):
        plan = dr.Plan(sc.geom, sc.wires, sc.edges, depth_form=form)
        info = plan.info()
        assert (info["kernel"], info["depth_form"]) == (kernel, want)
        unit = 2.0 ** -info["fixed_shift"]
        err = np.abs(plan.depths().cpu().numpy() - O.depths(sc.geom, sc.wires)).max()
        assert err < 4 * unit and abs(err - info["depth_err"]) < 1.5 * unit + 1e-12
        out = plan.reconstruct(torch.from_numpy(sc.images.view(np.int16)).cuda())
        torch.cuda.synchronize()
        assert_parity(out.cpu().numpy(), ref_of(sc), sc.images)


def test_climbing_wire_takes_the_exact_form():
    """A wire that also moves across the beam (eta != 0) has a remainder
    that depends on more than the wire's position along the beam: the plan
    keeps the exact form."""
    sc = synth.tiny_scan(8, rows=6, cols=40, K=25, roi_origin=(1000, 600), det_rows=2048,
                         det_cols=2048)
    sc.wires = synth.wire_path(25, dy=0.0002)
    plan = dr.Plan(sc.geom, sc.wires, sc.edges)
    assert plan.info()["depth_form"] == 0


def test_launch_shape_that_does_not_fit_is_reported():
    """A tile width given by the caller is a request for the running-sum
    kernels: when its tile does not fit in shared memory (801 steps x 256
    columns of images), dr_plan reports it instead of handing the scan to
    the interval kernel; without a given shape the plan picks a tile that
    fits."""
    geom = synth.detector_geometry(8, 256)
    wires = synth.wire_path(801)
    edges = synth.bin_edges(-400.0, 400.0, 1.0)
    with pytest.raises(dr.DrError) as e:
        dr.Plan(geom, wires, edges, tile_cols=256, bin_groups=2)
    assert e.value.status == 8  # DR_ERR_UNSUPPORTED
    plan = dr.Plan(geom, wires, edges)
    assert plan.info()["kernel"] == "rows"
    plan.close()
