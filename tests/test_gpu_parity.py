"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerance (stated with the method's workloads): every FP32 bin within
1e-4 x sum_k |dI_k| of its pixel, exactly 0 where the pixel never changes;
integer differences bit-exact; BF16 bins within 2^-8 of their magnitude
plus the FP32 bar.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2201_13309_gb300 import dr  # noqa: E402
from tests.gen import synth  # noqa: E402
from tests.golden.make_golden import odd_case, read_odd  # noqa: E402

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


def sum_abs_diff(images):
    return np.abs(np.diff(images.astype(np.int64), axis=0)).sum(0)


def assert_parity(got, ref, images, tol=FP32_TOL, rel=0.0):
    got = np.asarray(got, dtype=np.float64)
    s = sum_abs_diff(images)[None]
    err = np.abs(got - ref)
    bound = tol * s + rel * np.abs(ref)
    bad = err > bound
    assert not bad.any(), (
        f"{bad.sum()} bins off; worst err/sum|dI| = {(err / np.maximum(s, 1)).max():.3g}")
    assert np.all(got[np.broadcast_to(s == 0, got.shape)] == 0)
    return float((err / np.maximum(s, 1)).max())


def run(scan, **kw):
    plan = dr.Plan(scan.geom, scan.wires, scan.edges, **kw)
    out = plan.reconstruct(to_dev(scan.images))
    torch.cuda.synchronize()
    plan.check_device()
    return plan, out


def ref_of(scan, edge="leading"):
    return O.reconstruct(scan.geom, scan.wires, scan.images, scan.edges, edge)


def test_tiny_scan_rows_kernel():
    sc = synth.tiny_scan(0)
    plan, out = run(sc)
    info = plan.info()
    assert info["kernel"] == "rows" and info["pixels_per_thread"] == 4
    assert info["row_tables"] == 1
    assert_parity(out.cpu().numpy(), ref_of(sc), sc.images)


def test_odd_example_shape_golden():
    """Sec. III-B shape (4 images x 6 rows x 9 columns): odd width, plain
    loads, one pixel per thread, against the stored oracle values."""
    images, edges, expect = read_odd()
    sc, _ = odd_case()
    plan = dr.Plan(sc.geom, sc.wires, edges)
    assert plan.info()["pixels_per_thread"] == 1
    out = plan.reconstruct(to_dev(images))
    torch.cuda.synchronize()
    assert_parity(out.cpu().numpy(), expect, images)


def test_per_pixel_kernel_matches_rows_kernel_bitwise():
    sc = synth.tiny_scan(3)
    _, a = run(sc)
    plan, b = run(sc, force_pixels=True)
    assert plan.info()["kernel"] == "pixels"
    assert torch.equal(a.view(torch.int32), b.view(torch.int32))


def test_rotated_detector_per_pixel_depths():
    sc = synth.spot_scan(4, 24, 72, 33, 12, -60.0, 60.0, 1.0, rotate_deg=11.0,
                         tilt_deg=5.0, depth_range=(-0.03, 0.03))
    plan, out = run(sc)
    assert plan.info()["kernel"] == "pixels"
    assert_parity(out.cpu().numpy(), ref_of(sc), sc.images)


@pytest.fixture(scope="module", params=[280, 283])
def rotated_ragged(request):
    """Rotated detector whose width leaves a partial last tile for every tile
    width: 280 columns (TMA staging, 16-byte zero stores) and 283 (plain
    loads, scalar zero stores)."""
    sc = synth.spot_scan(6, 3, request.param, 37, 10, -60.0, 60.0, 0.7, rotate_deg=9.0,
                         tilt_deg=3.0, depth_range=(-0.03, 0.03))
    plan, out = run(sc)
    assert plan.info()["kernel"] == "pixels"
    assert_parity(out.cpu().numpy(), ref_of(sc), sc.images)
    return sc, out


@pytest.mark.parametrize("tc,bg", [(32, 16), (16, 32), (16, 16), (8, 64), (32, 8), (64, 8),
                                   (8, 1), (96, 4), (256, 2)])
def test_per_pixel_launch_shapes_agree(rotated_ragged, tc, bg):
    """Every tile width / share count gives bitwise the same bins, for full
    and partial slabs, vector and scalar zero stores."""
    sc, ref = rotated_ragged
    plan = dr.Plan(sc.geom, sc.wires, sc.edges, tile_cols=tc, bin_groups=bg)
    info = plan.info()
    assert (info["kernel"], info["tile_cols"], info["bin_groups"]) == ("pixels", tc, bg)
    out = plan.reconstruct(to_dev(sc.images))
    torch.cuda.synchronize()
    assert torch.equal(out.view(torch.int32), ref.view(torch.int32))


def _lit_scan(geom, wires, seed, lo_um, hi_um, width_um):
    rng = np.random.Generator(np.random.PCG64(seed))
    d = O.depths(geom, wires)
    scat = synth.Scatterers(rng.uniform(d.min(), d.max(), 4), rng.uniform(500.0, 5000.0, 4))
    images = synth.poisson_u16(rng, synth.expected_counts(geom, wires, scat, background=25.0))
    return synth.Scan(geom, wires, synth.bin_edges(lo_um, hi_um, width_um), images)


def test_wire_axis_oblique_to_beam():
    """Wire axis tilted 20 degrees toward the beam: the projected frame
    shrinks the beam by cos(angle) and detector rows no longer run along the
    axis (per-pixel depths)."""
    g = synth.detector_geometry(8, 48, roi_origin=(1000, 1000), det_rows=2048, det_cols=2048)
    a = np.deg2rad(20.0)
    g = dict(g, wire_axis=[np.cos(a), 0.0, np.sin(a)])
    sc = _lit_scan(g, synth.wire_path(41), 31, 0.0, 65.0, 1.0)
    plan, out = run(sc)
    assert plan.info()["kernel"] == "pixels"
    assert_parity(out.cpu().numpy(), ref_of(sc), sc.images)


def test_non_uniform_wire_steps():
    """Steps of 0.3 to 2 um drawn at random along the beam."""
    g = synth.detector_geometry(8, 64, roi_origin=(1000, 1000), det_rows=2048, det_cols=2048)
    rng = np.random.Generator(np.random.PCG64(32))
    z = np.cumsum(rng.uniform(0.3, 2.0, 41)) * 1e-3
    w = synth.wire_path(41)
    w[:, 2] = w[0, 2] + z - z[0]
    sc = _lit_scan(g, w, 33, 0.0, 70.0, 0.5)
    plan, out = run(sc)
    assert plan.info()["kernel"] == "rows"
    assert_parity(out.cpu().numpy(), ref_of(sc), sc.images)


@pytest.mark.parametrize("edge", ["leading", "trailing"])
def test_edges_and_reversed_travel(edge):
    sc = synth.tiny_scan(5, rows=16, cols=40, K=25)
    plan, out = run(sc, edge=edge)
    assert_parity(out.cpu().numpy(), ref_of(sc, edge), sc.images)
    back = synth.Scan(sc.geom, sc.wires[::-1].copy(), sc.edges, sc.images[::-1].copy())
    plan, out = run(back, edge=edge)
    assert plan.info()["reversed"] == 1
    assert_parity(out.cpu().numpy(), ref_of(back, edge), back.images)


def back_and_forth(n_up=24, n_down=10, n_up2=14):
    """Wire path along +z, back along -z, and on again (steps of 1 um)."""
    a = synth.wire_path(n_up)
    b = synth.wire_path(n_down + 1, z0=a[-1, 2], dz=-0.001)[1:]
    c = synth.wire_path(n_up2 + 1, z0=b[-1, 2], dz=0.001)[1:]
    return np.concatenate([a, b, c])


@pytest.mark.parametrize("edge", ["leading", "trailing", "both"])
@pytest.mark.parametrize("rotate", [0.0, 6.0])
def test_back_and_forth_wire_and_both_edges(edge, rotate):
    wires = back_and_forth()
    geom = synth.detector_geometry(12, 64, roi_origin=(26, 0), det_rows=64, det_cols=64,
                                   rotate_deg=rotate)
    rng = np.random.Generator(np.random.PCG64(81))
    scat = synth.tiny_scatterers(rng, 4)
    images = synth.poisson_u16(rng, synth.expected_counts(geom, wires, scat))
    sc = synth.Scan(geom, wires, synth.bin_edges(-40, 60, 1.0), images)
    plan, out = run(sc, edge=edge)
    info = plan.info()
    assert info["parts"] == 3 * (2 if edge == "both" else 1)
    assert info["kernel"] == ("pixels" if rotate else "rows")
    assert_parity(out.cpu().numpy(), ref_of(sc, edge), sc.images)


def test_both_edges_monotone_and_streamed():
    sc = synth.tiny_scan(82, rows=20, cols=64, K=41)
    plan, out = run(sc, edge="both")
    assert plan.info()["parts"] == 2
    assert_parity(out.cpu().numpy(), ref_of(sc, "both"), sc.images)
    h_img = torch.from_numpy(sc.images.view(np.int16)).pin_memory()
    h_out = torch.empty((sc.B, 20, 64)).pin_memory()
    ws = torch.empty(3 << 20, dtype=torch.uint8, device="cuda")
    plan.reconstruct_streamed(h_img, h_out, ws, slab_rows=3)
    torch.cuda.synchronize()
    assert torch.equal(h_out.view(torch.int32), out.cpu().view(torch.int32))


@pytest.mark.parametrize("H,W,K,lo,hi,w", [(5, 200, 37, -30, 30, 0.5),
                                           (3, 136, 9, -8, 8, 2.0),
                                           (7, 260, 51, -45, 45, 1.0),
                                           (2, 12, 3, -5, 5, 1.0)])
def test_ragged_tiles_and_bins(H, W, K, lo, hi, w):
    sc = synth.tiny_scan(H * W + K, rows=H, cols=W, K=K)
    sc.edges = synth.bin_edges(lo, hi, w)
    plan, out = run(sc)
    assert_parity(out.cpu().numpy(), ref_of(sc), sc.images)


def test_tile_overrides_agree_bitwise():
    sc = synth.tiny_scan(6, rows=8, cols=256, K=41)
    _, a = run(sc)
    for tc, bg in ((64, 1), (256, 2), (32, 8)):
        _, b = run(sc, tile_cols=tc, bin_groups=bg)
        assert torch.equal(a.view(torch.int32), b.view(torch.int32)), (tc, bg)


@pytest.mark.parametrize("tc", [8, 16, 32, 40, 64])
def test_small_tiles_multi_chunk(tc):
    """More than one TMA chunk of steps with narrow tiles (the chunk stride in
    shared memory must stay 128-byte aligned)."""
    sc = synth.tiny_scan(13, rows=3, cols=160, K=301, n_scat=3)
    sc.edges = synth.bin_edges(-40, 340, 2.0)
    _, a = run(sc)
    plan, b = run(sc, tile_cols=tc, bin_groups=2)
    info = plan.info()
    assert info["tma_chunks"] >= 2 and (info["tma_chunk"] * tc * 2) % 128 == 0
    assert torch.equal(a.view(torch.int32), b.view(torch.int32))
    assert_parity(b.cpu().numpy(), ref_of(sc), sc.images)


def test_autotuner_picks_a_valid_shape(tmp_path, monkeypatch):
    from paper_2201_13309_gb300 import autotune

    monkeypatch.setenv("DR_TUNE_CACHE", str(tmp_path / "tune.json"))
    sc = synth.tiny_scan(14, rows=8, cols=256, K=41)
    img = to_dev(sc.images)
    plan, best = autotune.tuned_plan(sc.geom, sc.wires, sc.edges, img, reps=2)
    assert not best["cached"] and len(best["candidates"]) >= 3
    out = plan.reconstruct(img)
    torch.cuda.synchronize()
    assert_parity(out.cpu().numpy(), ref_of(sc), sc.images)
    again = autotune.tune(sc.geom, sc.wires, sc.edges, img)
    assert again["cached"] and again["tile_cols"] == best["tile_cols"]


def test_sub_grid_steps():
    """Steps of 0.2 pm are below what FP32 geometry's position grid holds:
    the running-sum kernels refuse them and the interval kernel takes the
    scan, every interval with its depths in FP64; FP64 geometry takes them
    in the rows kernel."""
    sc = synth.tiny_scan(41, rows=4, cols=16, K=21)
    sc.wires = synth.wire_path(21, dz=2e-10)
    plan, out = run(sc)
    assert (plan.info()["kernel"], plan.info()["geom_precision"]) == ("intervals", 0)
    assert_parity(out.cpu().numpy(), ref_of(sc), sc.images)
    plan, out = run(sc, geom_precision="fp64")
    assert plan.info()["kernel"] == "rows"
    assert_parity(out.cpu().numpy(), ref_of(sc), sc.images, tol=1e-6)


def test_fp64_geometry_variant():
    sc = synth.tiny_scan(7)
    _, out = run(sc, geom_precision="fp64")
    err = assert_parity(out.cpu().numpy(), ref_of(sc), sc.images)
    assert err < 2e-6
    sc2 = synth.spot_scan(8, 16, 64, 21, 6, -40.0, 40.0, 1.0, rotate_deg=9.0,
                          depth_range=(-0.02, 0.02))
    _, out = run(sc2, geom_precision="fp64")
    assert_parity(out.cpu().numpy(), ref_of(sc2), sc2.images)


def test_bf16_output():
    sc = synth.tiny_scan(9)
    _, out = run(sc, out_dtype="bf16")
    assert out.dtype == torch.bfloat16
    assert_parity(out.float().cpu().numpy(), ref_of(sc), sc.images, rel=2.0 ** -8)


def test_differences_bit_exact():
    rng = np.random.Generator(np.random.PCG64(1))
    im = rng.integers(0, 65536, size=(9, 7, 33), dtype=np.uint16)
    got = dr.image_differences(to_dev(im)).cpu().numpy()
    assert np.array_equal(got.astype(np.int64), O.differences(im))


def test_gpu_depths_vs_oracle():
    sc = synth.spot_scan(2, 64, 48, 41, 4, -50, 50, 1.0, roi_origin=(0, 1000),
                         det_rows=2048, det_cols=2048)
    ref = O.depths(sc.geom, sc.wires)
    p32 = dr.Plan(sc.geom, sc.wires, sc.edges)
    d32 = p32.depths().cpu().numpy()
    p64 = dr.Plan(sc.geom, sc.wires, sc.edges, geom_precision="fp64")
    d64 = p64.depths().cpu().numpy()
    assert np.abs(d64 - ref).max() < 1e-12
    # FP32 geometry: fixed-point grid of 2^-shift mm plus FP32 remainder
    assert np.abs(d32 - ref).max() < 4.0 * 2.0 ** -p32.info()["fixed_shift"] + 1e-10


def test_gpu_depths_per_pixel_and_interval_plans():
    """dr_plan_depths for constants held per pixel (rotated detector) and for
    an interval plan (a wire climbing across the beam, travelling backwards),
    in the original step order."""
    rot = synth.spot_scan(3, 6, 40, 21, 4, -50, 50, 1.0, rotate_deg=7.0, tilt_deg=2.0)
    climb = synth.tiny_scan(4, rows=4, cols=24, K=30, roi_origin=(1900, 1000),
                            det_rows=2048, det_cols=2048)
    climb.wires = synth.wire_path(30, dy=0.005)[::-1].copy()
    # a wire moving across the beam (eta != 0) makes the FP32 remainder
    # ~eta * Z / D (0.05 mm here), taken with an approximate reciprocal of
    # D - eta: a few pm of error (measured 8.6 pm), 1e-5 of a 1 um step
    for sc, kernel, extra in ((rot, "pixels", 0.0), (climb, "intervals", 2e-8)):
        plan = dr.Plan(sc.geom, sc.wires, sc.edges)
        assert plan.info()["kernel"] == kernel
        ref = O.depths(sc.geom, sc.wires)
        got = plan.depths().cpu().numpy()
        assert np.abs(got - ref).max() < 4.0 * 2.0 ** -plan.info()["fixed_shift"] + 1e-10 + extra


def test_extreme_counts_and_constant_pixels():
    sc = synth.tiny_scan(10, rows=4, cols=64, K=17)
    im = sc.images.copy()
    im[:, 0, :8] = 65535
    im[::2, 1, :8] = 0
    im[1::2, 1, :8] = 65535
    im[:, 2, 8:16] = 777
    sc.images = im
    _, out = run(sc)
    got = out.cpu().numpy()
    assert_parity(got, ref_of(sc), im)
    assert np.all(got[:, 0, :8] == 0) and np.all(got[:, 2, 8:16] == 0)


def test_empty_roi_is_noop():
    sc = synth.tiny_scan(0, rows=4, cols=8, K=5)
    g = dict(sc.geom, rows=0)
    plan = dr.Plan(g, sc.wires, sc.edges)
    out = torch.empty((sc.B, 0, 8), device="cuda")
    plan.reconstruct(torch.empty((5, 0, 8), dtype=torch.int16, device="cuda"), out)
    torch.cuda.synchronize()


def test_deterministic_and_stream_async():
    sc = synth.tiny_scan(11)
    plan = dr.Plan(sc.geom, sc.wires, sc.edges)
    img = to_dev(sc.images)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        a = plan.reconstruct(img, stream=s)
        b = plan.reconstruct(img, stream=s)
    s.synchronize()
    assert torch.equal(a.view(torch.int32), b.view(torch.int32))


@pytest.mark.parametrize("kw", [{}, {"force_pixels": True}, {"force_intervals": True}])
def test_one_plan_on_two_streams_at_once(kw):
    """A plan is read-only after creation: the same plan on two streams with
    different images gives each stream's result bitwise as run alone."""
    sc = synth.tiny_scan(14, rows=24, cols=128, K=41)
    other = synth.tiny_scan(15, rows=24, cols=128, K=41).images
    plan = dr.Plan(sc.geom, sc.wires, sc.edges, **kw)
    a_img, b_img = to_dev(sc.images), to_dev(other)
    a_ref, b_ref = plan.reconstruct(a_img), plan.reconstruct(b_img)
    torch.cuda.synchronize()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    outs = []
    for _ in range(3):
        a_out, b_out = torch.empty_like(a_ref), torch.empty_like(b_ref)
        with torch.cuda.stream(s1):
            plan.reconstruct(a_img, a_out, stream=s1)
        with torch.cuda.stream(s2):
            plan.reconstruct(b_img, b_out, stream=s2)
        outs.append((a_out, b_out))
    torch.cuda.synchronize()
    plan.check_device()
    for a_out, b_out in outs:
        assert torch.equal(a_out.view(torch.int32), a_ref.view(torch.int32))
        assert torch.equal(b_out.view(torch.int32), b_ref.view(torch.int32))


def test_end_to_end_host_buffers():
    sc = synth.tiny_scan(12)
    plan = dr.Plan(sc.geom, sc.wires, sc.edges)
    h_img = torch.from_numpy(sc.images.view(np.int16)).pin_memory()
    h_out = torch.empty((sc.B, 64, 64), dtype=torch.float32).pin_memory()
    d_img = torch.empty_like(h_img, device="cuda")
    d_out = torch.empty_like(h_out, device="cuda")
    plan.reconstruct_host(h_img, h_out, d_img, d_out)
    torch.cuda.synchronize()
    ref = plan.reconstruct(to_dev(sc.images))
    torch.cuda.synchronize()
    assert torch.equal(h_out.view(torch.int32), ref.cpu().view(torch.int32))


def row_geometry(geom, r, nrows=1, cols=None):
    """The geometry of rows r .. r+nrows-1 of an ROI as an ROI of its own."""
    g = dict(geom)
    g["det_origin"] = (np.asarray(geom["det_origin"])
                       + r * np.asarray(geom["row_step"])).tolist()
    g["rows"] = nrows
    if cols is not None:
        g["cols"] = cols
    return g


def u16_int32(t):
    return t.to(torch.int32) & 0xFFFF


@pytest.mark.slow
def test_full_detector_sampled_rows():
    """2048x2048 pixels, 401 steps, 1001 bins, device-resident input, in the
    launch configuration the benchmark times; oracle on sampled rows, and
    conservation on every pixel whose depth range lies inside the bins."""
    spec = synth.full_scan_spec(0)
    img = synth.device_spot_images(spec.geom, spec.wires, spec.scat, 0, 20.0, "cuda")
    plan = dr.Plan(spec.geom, spec.wires, spec.edges)
    out = plan.reconstruct(img)
    torch.cuda.synchronize()
    plan.check_device()
    for r in (0, 1, 511, 1024, 1535, 2046, 2047):
        host = img[:, r:r + 1, :].cpu().numpy().view(np.uint16)
        ref = O.reconstruct(row_geometry(spec.geom, r), spec.wires, host, spec.edges)
        assert_parity(out[:, r:r + 1, :].cpu().numpy(), ref, host)
    d = O.depths(row_geometry(spec.geom, 0, 2048, cols=1), spec.wires)[:, 0, [0, -1]]
    inside = torch.from_numpy((d[:, 0] > spec.edges[0]) & (d[:, 1] < spec.edges[-1])).cuda()
    assert int(inside.sum()) > 1000
    for r0 in range(0, 2048, 256):
        blk = u16_int32(img[:, r0:r0 + 256, :])
        s = (blk[:-1] - blk[1:]).abs().sum(0).double()
        exp = (blk[0] - blk[-1]).double()
        tot = out[:, r0:r0 + 256, :].sum(0, dtype=torch.float64)
        err = (tot - exp).abs() - 1e-4 * s
        sel = err[inside[r0:r0 + 256]]
        if sel.numel():
            assert float(sel.max()) <= 0.0


@pytest.mark.slow
def test_maximum_size_sampled_rows():
    """The largest scan shape the uneven batch draws: 2048x2048 pixels, 801
    steps, 1601 bins of 0.5 um (6.7 GB in, 26.9 GB out)."""
    spec = synth.full_scan_spec(3)
    spec.wires = synth.wire_path(801)
    spec.edges = synth.bin_edges(-400.0, 400.0, 0.5)
    img = synth.device_spot_images(spec.geom, spec.wires, spec.scat, 3, 20.0, "cuda")
    plan = dr.Plan(spec.geom, spec.wires, spec.edges)
    out = plan.reconstruct(img)
    torch.cuda.synchronize()
    plan.check_device()
    for r in (0, 700, 1500, 2047):
        host = img[:, r:r + 1, :].cpu().numpy().view(np.uint16)
        ref = O.reconstruct(row_geometry(spec.geom, r), spec.wires, host, spec.edges)
        assert_parity(out[:, r:r + 1, :].cpu().numpy(), ref, host)
    del out, img
    torch.cuda.empty_cache()


@pytest.mark.parametrize("K,rotate,climb", [(2049, 0.0, False), (4300, 9.0, False),
                                            (2600, 0.0, True)])
def test_long_scans_in_parts(K, rotate, climb):
    """Runs longer than 2048 steps are cut into parts that share their end
    steps (the images of a tile are staged for all the steps of a part);
    later parts add to the output.  Rows, per-pixel and interval kernels."""
    rng = np.random.Generator(np.random.PCG64(K))
    geom = synth.detector_geometry(3, 16, roi_origin=(1500, 900), det_rows=2048,
                                   det_cols=2048, rotate_deg=rotate)
    wires = synth.wire_path(K, dz=1e-4)
    if climb:
        wires[:, 1] += np.arange(K) * 0.00035 + rng.normal(0.0, 0.00004, K)
    d = O.depths(geom, wires)
    scat = synth.Scatterers(rng.uniform(d.min(), d.max(), 3), rng.uniform(500.0, 5000.0, 3))
    images = synth.poisson_u16(rng, synth.expected_counts(geom, wires, scat, background=20.0))
    sc = synth.Scan(geom, wires, synth.bin_edges(np.floor(d.min() * 1e3) - 2,
                                                 np.ceil(d.max() * 1e3) + 2, 2.0), images)
    plan, out = run(sc)
    info = plan.info()
    assert info["parts"] == -(-(K - 1) // 2047)
    assert info["kernel"] == ("intervals" if climb else "pixels" if rotate else "rows")
    assert_parity(out.cpu().numpy(), ref_of(sc), sc.images)
