"""Persistent batched launch (one kernel for many uneven scans, replayed from
a CUDA graph) against the per-scan launches and the FP64 oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2201_13309_gb300 import dr  # noqa: E402
from tests.gen import synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()


def _dev(images):
    return torch.from_numpy(np.ascontiguousarray(images).view(np.int16)).cuda()


def _scans():
    a = synth.tiny_scan(31, rows=40, cols=256, K=61)
    b = synth.tiny_scan(32, rows=8, cols=512, K=301, n_scat=2)
    b.edges = synth.bin_edges(-100.0, 320.0, 2.0)
    c = synth.tiny_scan(33, rows=24, cols=64, K=37)
    c.edges = synth.bin_edges(-30.0, 60.0, 0.5)
    d = synth.tiny_scan(34, rows=16, cols=128, K=45)
    d = synth.Scan(d.geom, d.wires[::-1].copy(), d.edges, d.images[::-1].copy())
    return [(a, "leading"), (b, "leading"), (c, "trailing"), (d, "leading")]


def test_batch_matches_per_scan_launches_bitwise():
    jobs, refs, keep = [], [], []
    for sc, edge in _scans():
        plan = dr.Plan(sc.geom, sc.wires, sc.edges, edge=edge)
        img = _dev(sc.images)
        refs.append(plan.reconstruct(img))
        out = torch.full_like(refs[-1], float("nan"))
        jobs.append((plan, img, out))
        keep.append((sc, edge))
    batch = dr.Batch(jobs)
    info = batch.info()
    assert info["scans"] == 4 and info["threads"] == 512 and info["items"] > 0
    batch.launch()
    torch.cuda.synchronize()
    batch.check_device()
    for (plan, img, out), ref in zip(jobs, refs):
        assert torch.equal(out.view(torch.int32), ref.view(torch.int32))
    # one against the oracle directly
    sc, edge = keep[2]
    got = jobs[2][2].cpu().numpy().astype(np.float64)
    want = O.reconstruct(sc.geom, sc.wires, sc.images, sc.edges, edge)
    s = np.abs(np.diff(sc.images.astype(np.int64), axis=0)).sum(0)[None]
    assert np.all(np.abs(got - want) <= 1e-4 * s)


def test_one_shot_batch_reconstruct():
    """dr_batch_reconstruct (create, launch, wait, check, destroy in one call)
    gives the per-scan results bitwise."""
    jobs, refs = [], []
    for sc, edge in _scans():
        plan = dr.Plan(sc.geom, sc.wires, sc.edges, edge=edge)
        img = _dev(sc.images)
        refs.append(plan.reconstruct(img))
        jobs.append((plan, img, torch.full_like(refs[-1], float("nan"))))
    dr.batch_reconstruct(jobs)
    for (_, _, out), ref in zip(jobs, refs):
        assert torch.equal(out.view(torch.int32), ref.view(torch.int32))


@pytest.mark.parametrize("per_sm,cap,nt", [(2, 0, 512), (2, 64, 512), (1, 32, 512), (1, 0, 256),
                                           (2, 0, 256)])
def test_batch_modes_agree(per_sm, cap, nt):
    jobs, refs = [], []
    for sc, edge in _scans():
        plan = dr.Plan(sc.geom, sc.wires, sc.edges, edge=edge)
        img = _dev(sc.images)
        refs.append(plan.reconstruct(img))
        jobs.append((plan, img, torch.full_like(refs[-1], float("nan"))))
    batch = dr.Batch(jobs, ctas_per_sm=per_sm, max_tile_cols=cap, threads=nt)
    assert batch.info()["threads"] == nt
    batch.launch()
    torch.cuda.synchronize()
    for (_, _, out), ref in zip(jobs, refs):
        assert torch.equal(out.view(torch.int32), ref.view(torch.int32))


def test_batch_autotuner():
    from paper_2201_13309_gb300 import autotune

    jobs, refs = [], []
    for sc, edge in _scans()[:2]:
        plan = dr.Plan(sc.geom, sc.wires, sc.edges, edge=edge)
        img = _dev(sc.images)
        refs.append(plan.reconstruct(img))
        jobs.append((plan, img, torch.empty_like(refs[-1])))
    batch, tune = autotune.tuned_batch(jobs, reps=1)
    assert len(tune["candidates"]) >= 2
    batch.launch()
    torch.cuda.synchronize()
    for (_, _, out), ref in zip(jobs, refs):
        assert torch.equal(out.view(torch.int32), ref.view(torch.int32))


def test_batch_replay_with_new_images():
    sc, _ = _scans()[0]
    plan = dr.Plan(sc.geom, sc.wires, sc.edges)
    img = _dev(sc.images)
    out = plan.empty_output()
    batch = dr.Batch([(plan, img, out)])
    batch.launch()
    other = synth.tiny_scan(99, rows=40, cols=256, K=61).images
    img.copy_(_dev(other))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    batch.launch(stream=s)
    s.synchronize()
    ref = plan.reconstruct(_dev(other))
    torch.cuda.synchronize()
    assert torch.equal(out.view(torch.int32), ref.view(torch.int32))


def _rotated_scans():
    """Scans on a rotated (and tilted) detector: every pixel has its own
    depth sequence, so their plans take the per-pixel kernel; one with bins
    wider than its steps (more than one step per bin)."""
    a = synth.spot_scan(41, 12, 96, 45, 8, -60.0, 60.0, 1.0, rotate_deg=10.0,
                        depth_range=(-0.03, 0.03))
    b = synth.spot_scan(42, 6, 200, 33, 6, -50.0, 60.0, 2.0, rotate_deg=-7.0, tilt_deg=4.0,
                        depth_range=(-0.03, 0.03))
    c = synth.spot_scan(43, 9, 64, 61, 6, -60.0, 80.0, 0.5, rotate_deg=3.0,
                        depth_range=(-0.03, 0.03))
    return [(a, "leading"), (b, "leading"), (c, "trailing")]


@pytest.mark.parametrize("per_sm,nt", [(1, 512), (2, 512), (1, 256), (3, 512)])
def test_batch_of_rows_and_per_pixel_plans(per_sm, nt):
    """Rows and per-pixel tiles in one persistent launch: every scan bitwise
    as its own launch, and each per-pixel scan against the FP64 oracle."""
    jobs, refs, keep = [], [], []
    for sc, edge in _scans()[:2] + _rotated_scans():
        plan = dr.Plan(sc.geom, sc.wires, sc.edges, edge=edge)
        img = _dev(sc.images)
        refs.append(plan.reconstruct(img))
        jobs.append((plan, img, torch.full_like(refs[-1], float("nan"))))
        keep.append((sc, edge, plan.info()))
    kinds = [k[2]["kernel"] for k in keep]
    assert kinds == ["rows", "rows", "pixels", "pixels", "pixels"]
    assert [k[2]["one_step_per_bin"] for k in keep[2:]] == [1, 0, 1]
    batch = dr.Batch(jobs, ctas_per_sm=per_sm, threads=nt)
    batch.launch()
    torch.cuda.synchronize()
    batch.check_device()
    for (_, _, out), ref in zip(jobs, refs):
        assert torch.equal(out.view(torch.int32), ref.view(torch.int32))
    for (sc, edge, _), (_, _, out) in zip(keep[2:], jobs[2:]):
        want = O.reconstruct(sc.geom, sc.wires, sc.images, sc.edges, edge)
        s = np.abs(np.diff(sc.images.astype(np.int64), axis=0)).sum(0)[None]
        assert np.all(np.abs(out.cpu().numpy().astype(np.float64) - want) <= 1e-4 * s)


def test_batch_rejects_unsupported_jobs():
    sc = synth.tiny_scan(35, rows=4, cols=64, K=9)
    for kw in ({"geom_precision": "fp64"}, {"geom_precision": "fp64", "force_pixels": True}):
        pix = dr.Plan(sc.geom, sc.wires, sc.edges, **kw)
        img = _dev(sc.images)
        with pytest.raises(dr.DrError) as ex:
            dr.Batch([(pix, img, pix.empty_output())])
        assert ex.value.status == 8 and "FP64" in str(ex.value)
    odd = synth.tiny_scan(36, rows=4, cols=12, K=9)
    p2 = dr.Plan(odd.geom, odd.wires, odd.edges)
    with pytest.raises(dr.DrError):
        dr.Batch([(p2, _dev(odd.images), p2.empty_output())])


def test_batch_with_interval_plans():
    """Interval-kernel plans (a wire climbing across the beam with jitter;
    one forced on a rotated detector) batched with rows and per-pixel plans:
    bitwise the per-scan launches (the integer sums of a bin do not depend on
    the window the batch's budget gives), and against the oracle."""
    rng = np.random.Generator(np.random.PCG64(37))
    geom = synth.detector_geometry(6, 40, roi_origin=(1900, 1000), det_rows=2048, det_cols=2048)
    wires = synth.wire_path(41, dy=0.0035)
    wires[:, 1] += rng.normal(0.0, 0.0004, 41)
    d = O.depths(geom, wires)
    scat = synth.Scatterers(rng.uniform(d.min(), d.max(), 4), rng.uniform(500.0, 5000.0, 4))
    images = synth.poisson_u16(rng, synth.expected_counts(geom, wires, scat, background=30.0))
    climb = synth.Scan(geom, wires,
                       synth.bin_edges(np.floor(d.min() * 1e3) - 2, np.ceil(d.max() * 1e3) + 2,
                                       0.5), images)
    rot = synth.spot_scan(38, 5, 96, 37, 6, -60.0, 60.0, 0.7, rotate_deg=9.0,
                          depth_range=(-0.03, 0.03))
    cases = [(climb, {}), (rot, {"force_intervals": True}), (_scans()[0][0], {}), (rot, {})]
    jobs, refs = [], []
    for sc, kw in cases:
        plan = dr.Plan(sc.geom, sc.wires, sc.edges, **kw)
        img = _dev(sc.images)
        refs.append(plan.reconstruct(img))
        jobs.append((plan, img, torch.full_like(refs[-1], float("nan"))))
    kinds = [p.info()["kernel"] for p, _, _ in jobs]
    assert kinds == ["intervals", "intervals", "rows", "pixels"]
    for per_sm in (1, 2, 3):  # (3: the interval tiles' bin window shrinks to 75 KB)
        batch = dr.Batch(jobs, ctas_per_sm=per_sm)
        batch.launch()
        torch.cuda.synchronize()
        batch.check_device()
        for (_, _, out), ref in zip(jobs, refs):
            assert torch.equal(out.view(torch.int32), ref.view(torch.int32))
        batch.close()
    for (sc, _), (_, _, out) in zip(cases[:2], jobs[:2]):
        want = O.reconstruct(sc.geom, sc.wires, sc.images, sc.edges)
        s = np.abs(np.diff(sc.images.astype(np.int64), axis=0)).sum(0)[None]
        assert np.all(np.abs(out.cpu().numpy().astype(np.float64) - want) <= 1e-4 * s)
