"""Pins of the FP64 oracle to facts outside itself (CPU only).

Each pin checks the oracle against something it does not compute itself:
brute-force ray-cylinder occlusion from the forward model, the exact
quadratic solution of the tangent condition, the far-detector limit, fine
subdivision of the depth intervals, conservation of the total intensity
change, rigid-motion invariance, invariance to the lengths of the direction
vectors and the sense of the wire axis, and noise-free forward-model scans.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from tests.gen import synth as S

R = S.WIRE_R_MM
YW = S.WIRE_Y_MM


def _single_pixel_geom(x, y, z):
    g = S.detector_geometry(1, 1)
    g["det_origin"] = [x, y, z]
    return g


def _leading_boundary_bisect(q, centre, axis=(1.0, 0.0, 0.0), radius=R,
                             beam_o=(0.0, 0.0, 0.0), beam_d=(0.0, 0.0, 1.0)):
    """Upper end of the set of beam depths hidden from pixel q (bisection on
    the forward model's brute-force occlusion predicate)."""
    bo = np.asarray(beam_o, float)
    bd = np.asarray(beam_d, float)
    bd = bd / np.linalg.norm(bd)
    qa = np.asarray(q, float)[None, :]

    def hidden(d):
        return bool(S.hidden_by_wire(bo + d * bd, qa, centre, axis, radius)[0])

    grid = np.arange(-3.0, 3.0, 2e-4)
    hid = S.hidden_by_wire(bo[None, :] + grid[:, None] * bd[None, :], qa, centre, axis, radius)
    assert hid.any(), "wire hides nothing from this pixel"
    i = int(np.nonzero(hid)[0].max())
    a, b = grid[i], grid[i] + 2e-4
    assert hidden(a) and not hidden(b)
    for _ in range(80):
        m = 0.5 * (a + b)
        if hidden(m):
            a = m
        else:
            b = m
    return 0.5 * (a + b)


def _quadratic_depths(Y, Z, y, z, radius=R):
    """Both roots of (a t - b)^2 = R^2 (Y^2 + (Z - t)^2), a = Y - y,
    b = zY - Zy: the lines through (Y, Z) tangent to the circle (y, z; R)
    meet the beam (y = 0) at depth t.  Returns (leading(+R), trailing(-R))."""
    a = Y - y
    b = z * Y - Z * y
    A = a * a - radius * radius
    Bq = 2.0 * radius * radius * Z - 2.0 * a * b
    C = b * b - radius * radius * (Y * Y + Z * Z)
    disc = math.sqrt(Bq * Bq - 4.0 * A * C)
    q = -0.5 * (Bq + math.copysign(disc, Bq))
    roots = [q / A, C / q]
    lead = [t for t in roots if a * t - b > 0]
    trail = [t for t in roots if a * t - b < 0]
    assert len(lead) == 1 and len(trail) == 1
    return lead[0], trail[0]


CASES = [(0.0, 0.0, -0.020), (0.0, 6.3, -0.020), (0.0, -6.3, 0.0),
         (0.0, 204.7, -0.020), (3.1, -204.7, 0.380), (-150.0, 100.0, 0.125)]


@pytest.mark.parametrize("x,Z,zc", CASES)
def test_depth_vs_bruteforce_occlusion(x, Z, zc):
    q = (x, S.DET_Y_MM, Z)
    wires = np.array([[0.0, YW, zc], [0.0, YW, zc + 0.001]])
    d = O.depths(_single_pixel_geom(*q), wires)[0, 0, 0]
    ref = _leading_boundary_bisect(q, wires[0])
    assert abs(d - ref) < 1e-10, (d, ref)


@pytest.mark.parametrize("x,Z,zc", CASES)
def test_depth_vs_quadratic_closed_form(x, Z, zc):
    q = (x, S.DET_Y_MM, Z)
    wires = np.array([[0.0, YW, zc], [0.0, YW, zc + 0.001]])
    g = _single_pixel_geom(*q)
    lead = O.depths(g, wires, "leading")[0, 0, 0]
    trail = O.depths(g, wires, "trailing")[0, 0, 0]
    ql, qt = _quadratic_depths(S.DET_Y_MM, Z, YW, zc)
    assert abs(lead - ql) < 1e-12
    assert abs(trail - qt) < 1e-12
    assert trail < lead


def test_spot_values_from_closed_form():
    # leading edge, wire at z = -20 um: centre pixel and a far edge pixel
    for Z, expect_um in ((0.0, 6.005888), (204.7, -192.855553)):
        g = _single_pixel_geom(0.0, S.DET_Y_MM, Z)
        w = np.array([[0.0, YW, -0.020], [0.0, YW, -0.019]])
        d_um = O.depths(g, w)[0, 0, 0] * 1e3
        assert abs(d_um - expect_um) < 2e-6, d_um


def test_far_detector_limit():
    # a pixel infinitely far along y sees the wire edge at z + R
    for zc in (-0.02, 0.0, 0.3):
        g = _single_pixel_geom(0.0, 1e9, 0.0)
        w = np.array([[0.0, YW, zc], [0.0, YW, zc + 0.001]])
        assert abs(O.depths(g, w)[0, 0, 0] - (zc + R)) < 1e-9
        assert abs(O.depths(g, w, "trailing")[0, 0, 0] - (zc - R)) < 1e-9


def test_wire_moving_backwards_swaps_edges():
    # travelling toward -z, the leading edge is the lower end
    g = _single_pixel_geom(0.0, S.DET_Y_MM, 1.0)
    fwd = np.array([[0.0, YW, 0.0], [0.0, YW, 0.001]])
    bwd = fwd[::-1].copy()
    lf = O.depths(g, fwd, "leading")[0, 0]
    tb = O.depths(g, bwd, "trailing")[0, 0]
    assert np.allclose(lf, tb[::-1], atol=0, rtol=0)
    assert O.depths(g, bwd, "leading")[0, 0, 0] < tb[0]


def _random_rotation(rng):
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def test_rigid_motion_invariance():
    """Depths are lengths along the beam: a rotation plus translation of the
    whole set-up (beam, wire, detector) must not change them."""
    rng = np.random.Generator(np.random.PCG64(7))
    geom = S.detector_geometry(5, 7, rotate_deg=17.0, tilt_deg=-8.0)
    geom["det_origin"] = (np.asarray(geom["det_origin"]) + [0, 0, 30.0]).tolist()
    wires = S.wire_path(9)
    ref = O.depths(geom, wires)
    for _ in range(3):
        Rm = _random_rotation(rng)
        t = rng.normal(size=3) * 50.0
        g2 = dict(geom)
        for key in ("beam_dir", "row_step", "col_step", "wire_axis"):
            g2[key] = (Rm @ np.asarray(geom[key])).tolist()
        for key in ("beam_origin", "det_origin"):
            g2[key] = (Rm @ np.asarray(geom[key]) + t).tolist()
        w2 = wires @ Rm.T + t
        assert np.allclose(O.depths(g2, w2), ref, atol=1e-12, rtol=0)


def test_depth_scales_with_beam_obliquity():
    """A beam inclined in the plane of the wire axis: the projected geometry
    is unchanged, so depths along the beam grow by 1/cos(angle)."""
    geom = S.detector_geometry(3, 4)
    wires = S.wire_path(5)
    ref = O.depths(geom, wires)
    ang = math.radians(25.0)
    g2 = dict(geom)
    g2["beam_dir"] = [math.sin(ang), 0.0, math.cos(ang)]
    assert np.allclose(O.depths(g2, wires) * math.cos(ang), ref, atol=1e-13, rtol=0)


def test_differences_exact():
    rng = np.random.Generator(np.random.PCG64(3))
    im = rng.integers(0, 65536, size=(7, 3, 5), dtype=np.uint16)
    d = O.differences(im)
    assert d.dtype == np.int64
    assert np.array_equal(d, im[:-1].astype(np.int64) - im[1:].astype(np.int64))
    assert d.min() < -30000 and d.max() > 30000


def _subdivided(depth_seq, images, edges, edge="leading", n=20000):
    """Brute-force apportioning: each interval cut into n equal pieces whose
    share of the difference is dropped into the bin holding the piece's
    midpoint."""
    P, K = depth_seq.shape
    B = edges.shape[0] - 1
    out = np.zeros((B, P))
    frac = (np.arange(n) + 0.5) / n
    for p in range(P):
        for k in range(K - 1):
            a, b = int(images[k, p]), int(images[k + 1, p])
            dI = a - b if edge == "leading" else b - a
            x = depth_seq[p, k] + frac * (depth_seq[p, k + 1] - depth_seq[p, k])
            h, _ = np.histogram(x, bins=edges)
            out[:, p] += dI * h / n
    return out


def test_apportion_vs_fine_subdivision():
    rng = np.random.Generator(np.random.PCG64(11))
    P, K = 6, 9
    steps = rng.uniform(0.2, 2.0, size=(P, K - 1))
    d = np.cumsum(np.concatenate([rng.uniform(-3, 0, (P, 1)), steps], 1), 1)
    d[3] = d[3][::-1].copy()                     # a decreasing sequence
    d[4, 4:] = d[4, 4:] - 5.0                    # a non-monotone one
    edges = np.sort(rng.uniform(-4.0, 10.0, 23))  # uneven bins
    images = rng.integers(0, 5000, size=(K, P), dtype=np.uint16)
    for edge in ("leading", "trailing"):
        got = O.apportion(d, images, edges, edge)
        ref = _subdivided(d, images, edges, edge)
        tol = 4.0 * np.abs(np.diff(images.astype(np.int64), axis=0)).sum() / 20000
        assert np.abs(got - ref).max() < tol


def test_apportion_zero_length_interval_and_edges():
    edges = np.array([0.0, 1.0, 2.0, 3.0])
    d = np.array([[0.5, 1.0, 1.0, 2.5, 3.5]])      # interval 1 has zero length
    images = np.array([[100], [90], [60], [50], [0]], dtype=np.uint16)
    out = O.apportion(d, images, edges)[:, 0]
    # k=0: 10 over [0.5, 1) -> bin 0; k=1: 30 at x = 1 -> bin 1 ([1, 2));
    # k=2: 10 over [1, 2.5) -> 1/1.5 of it to bin 1 and 0.5/1.5 to bin 2;
    # k=3: 50 over [2.5, 3.5) -> half to bin 2, half dropped above e_B
    exp = np.array([10.0, 30.0 + 10.0 / 1.5, 10.0 * 0.5 / 1.5 + 25.0])
    assert np.allclose(out, exp, rtol=0, atol=1e-12)


def _inside_rows(scan, d):
    return [r for r in range(scan.geom["rows"])
            if d[r, 0, 0] > scan.edges[0] and d[r, 0, -1] < scan.edges[-1]]


def test_conservation_tiny_scan():
    sc = S.tiny_scan(0)
    d = O.depths(sc.geom, sc.wires)
    rows = _inside_rows(sc, d)
    assert len(rows) > 20
    out = O.reconstruct(sc.geom, sc.wires, sc.images, sc.edges)
    tot = out.sum(0)
    exp = sc.images[0].astype(np.int64) - sc.images[-1].astype(np.int64)
    sabs = np.abs(np.diff(sc.images.astype(np.int64), axis=0)).sum(0)
    err = np.abs(tot[rows] - exp[rows]) / np.maximum(sabs[rows], 1)
    assert err.max() < 1e-12


def test_constant_offset_and_linearity():
    sc = S.tiny_scan(1, rows=6, cols=9, K=12)
    base = O.reconstruct(sc.geom, sc.wires, sc.images, sc.edges)
    const = np.full_like(sc.images, 1234)
    assert np.array_equal(O.reconstruct(sc.geom, sc.wires, const, sc.edges),
                          np.zeros_like(base))
    shifted = (sc.images.astype(np.int64) + 777).astype(np.uint16)
    assert np.array_equal(O.reconstruct(sc.geom, sc.wires, shifted, sc.edges), base)
    other = S.tiny_scan(2, rows=6, cols=9, K=12).images
    both = (sc.images.astype(np.int64) + other).astype(np.uint16)
    lin = base + O.reconstruct(sc.geom, sc.wires, other, sc.edges)
    assert np.allclose(O.reconstruct(sc.geom, sc.wires, both, sc.edges), lin,
                       rtol=0, atol=1e-9)


def test_noise_free_scatterer_lands_in_its_interval():
    """Forward model with one scatterer, no noise: the leading edge hides it
    between steps k*-1 and k*, so +A must land on [d_{k*-1}, d_{k*}], which
    has to contain the scatterer depth; the reveal by the trailing edge puts
    -A on the leading-edge interval of that step."""
    geom = S.detector_geometry(3, 2, roi_origin=(30, 0), det_rows=64, det_cols=64)
    wires = S.wire_path(41)
    A = 1000.0
    for s in (0.0101, 0.0154, 0.0233, 0.0309):
        scat = S.Scatterers(np.array([s]), np.array([A]))
        images = np.rint(S.expected_counts(geom, wires, scat)).astype(np.uint16)
        d = O.depths(geom, wires)
        out = O.reconstruct(geom, wires, images, S.bin_edges(-50, 50, 1.0))
        for r in range(3):
            vis = images[:, r, 0] > 0
            kstar = int(np.argmin(vis))          # first hidden step
            assert vis[:kstar].all() and kstar > 0
            assert d[r, 0, kstar - 1] <= s <= d[r, 0, kstar]
            dI = -np.diff(images[:, r, 0].astype(np.int64))
            assert dI[kstar - 1] == A
            if (~vis[kstar:]).all():
                assert out[:, r, 0].sum() == pytest.approx(A, abs=1e-9)
            lo, hi = d[r, 0, kstar - 1], d[r, 0, kstar]
            e = S.bin_edges(-50, 50, 1.0)
            jlo = np.searchsorted(e, lo, "right") - 1
            jhi = np.searchsorted(e, hi, "right") - 1
            js = np.searchsorted(e, s, "right") - 1
            assert jlo <= js <= jhi
            band = out[jlo:jhi + 1, r, 0]
            assert band.sum() == pytest.approx(A, abs=1e-9) or (~vis[kstar:]).sum() < 41


def test_tiny_scan_peaks_at_scatterer_depths():
    """Noisy 64x64 scan: summed over a row (all pixels of a row share their
    depths), each scatterer that the leading edge sweeps past shows up as a
    peak within one bin of its true depth holding its full intensity."""
    sc = S.tiny_scan(0)
    d = O.depths(sc.geom, sc.wires)
    out = O.reconstruct(sc.geom, sc.wires, sc.images, sc.edges)
    e = sc.edges
    W = sc.geom["cols"]
    checked = 0
    for r in range(0, 64, 3):
        prof = out[:, r, :].sum(1)
        for s, A in zip(sc.scat.depth, sc.scat.peak):
            if not (d[r, 0, 0] + 0.002 < s < d[r, 0, -1] - 0.002):
                continue
            js = int(np.searchsorted(e, s, "right") - 1)
            win = prof[js - 2:js + 3]
            assert abs(int(np.argmax(win)) - 2) <= 1
            mass = prof[js - 1:js + 2].sum()
            sigma = math.sqrt(W * 2 * (sc.scat.peak.sum()))
            assert abs(mass - W * A) < 5 * sigma + 0.05 * W * A
            checked += 1
    assert checked >= 15


def test_trailing_edge_conservation_tiny_scan():
    """The trailing edge reveals what the leading edge hid: its differences
    are I_{k+1} - I_k, so wherever a pixel's whole trailing-edge sweep lies
    inside the bins, the bins sum to I_last - I_first."""
    sc = S.tiny_scan(0)
    d = O.depths(sc.geom, sc.wires, "trailing")
    rows = _inside_rows(sc, d)
    assert len(rows) > 20
    out = O.reconstruct(sc.geom, sc.wires, sc.images, sc.edges, edge="trailing")
    tot = out.sum(0)
    exp = sc.images[-1].astype(np.int64) - sc.images[0].astype(np.int64)
    sabs = np.abs(np.diff(sc.images.astype(np.int64), axis=0)).sum(0)
    err = np.abs(tot[rows] - exp[rows]) / np.maximum(sabs[rows], 1)
    assert err.max() < 1e-12
    assert np.abs(exp[rows]).max() > 100          # the sums are not all zero


def test_noise_free_scatterer_revealed_by_trailing_edge():
    """Forward model with one scatterer that starts hidden (between the two
    tangents at step 0), no noise: the trailing edge uncovers it between the
    brute-force steps k-1 (hidden) and k (visible).  The trailing-edge
    reconstruction must put exactly +A on the trailing interval
    [d_{k-1}, d_k], which contains the scatterer depth, and nothing
    elsewhere."""
    geom = S.detector_geometry(3, 2, roi_origin=(30, 0), det_rows=64, det_cols=64)
    wires = S.wire_path(41)
    e = S.bin_edges(-50, 50, 1.0)
    A = 1000.0
    d = O.depths(geom, wires, "trailing")
    for s in (-0.0351, -0.0254, -0.0187, -0.0109):
        scat = S.Scatterers(np.array([s]), np.array([A]))
        images = np.rint(S.expected_counts(geom, wires, scat)).astype(np.uint16)
        out = O.reconstruct(geom, wires, images, e, edge="trailing")
        for r in range(3):
            vis = images[:, r, 0] > 0
            kr = int(np.argmax(vis))                 # first visible step
            assert kr > 0 and not vis[:kr].any() and vis[kr:].all()
            lo, hi = d[r, 0, kr - 1], d[r, 0, kr]
            assert lo <= s <= hi
            jlo = int(np.searchsorted(e, lo, "right") - 1)
            jhi = int(np.searchsorted(e, hi, "right") - 1)
            col = out[:, r, 0]
            band = col[jlo:jhi + 1]
            assert band.sum() == pytest.approx(A, abs=1e-9)
            assert (band >= 0).all() and band.max() > 0.4 * A
            assert np.abs(col).sum() == pytest.approx(A, abs=1e-9)


def test_both_edges_hand_computed():
    """One pixel far along y, three wire steps: the leading edge sits at
    z_k + R and the trailing edge at z_k - R (the far-detector limit).  With
    I = (100, 70, 60) the leading differences are +30, +10 and the trailing
    ones -30, -10; each interval is 1 um long and straddles two 1 um bins
    half and half.  The both-edge result is the mean of the two."""
    g = _single_pixel_geom(0.0, 1e9, 0.0)
    w = np.array([[0.0, YW, 0.0], [0.0, YW, 0.001], [0.0, YW, 0.002]])
    images = np.array([100, 70, 60], dtype=np.uint16).reshape(3, 1, 1)
    e = np.array([-26.5, -25.5, -24.5, -23.5, 25.5, 26.5, 27.5, 28.5]) * 1e-3
    lead = np.array([0, 0, 0, 0, 15, 20, 5], float)
    trail = np.array([-15, -20, -5, 0, 0, 0, 0], float)
    got_l = O.reconstruct(g, w, images, e, "leading")[:, 0, 0]
    got_t = O.reconstruct(g, w, images, e, "trailing")[:, 0, 0]
    got_b = O.reconstruct(g, w, images, e, "both")[:, 0, 0]
    tol = 1e-4                 # depths within 1e-9 mm of z +- R: 1e-6 of a bin
    assert np.abs(got_l - lead).max() < tol
    assert np.abs(got_t - trail).max() < tol
    assert np.abs(got_b - 0.5 * (lead + trail)).max() < tol


def test_depths_do_not_depend_on_direction_lengths_or_axis_sense():
    """The beam and the wire axis enter as directions only: scaling either
    vector, or reversing the wire axis (the same line), leaves every depth of
    both edges unchanged.  A rotated, tilted detector with an oblique wire
    axis and an oblique beam, so that no component is trivially zero."""
    g = S.detector_geometry(4, 5, rotate_deg=7.0, tilt_deg=4.0)
    g["wire_axis"] = [1.0, 0.05, -0.03]
    g["beam_dir"] = [0.02, 0.01, 1.0]
    wires = S.wire_path(9)
    base = {e: O.depths(g, wires, e) for e in ("leading", "trailing")}
    assert not np.allclose(base["leading"], base["trailing"])
    for key, f in (("beam_dir", 2.5), ("beam_dir", 0.01), ("wire_axis", 0.3),
                   ("wire_axis", -1.0), ("wire_axis", -4.0)):
        h = dict(g)
        h[key] = [f * v for v in g[key]]
        for e in base:
            got = O.depths(h, wires, e)
            assert np.abs(got - base[e]).max() < 1e-10, (key, f, e)


def test_leading_edge_follows_the_net_travel():
    """A path whose first step goes backwards (0.4 of a step) before the
    forward sweep.  The leading edge is the end that moves with the wire's
    net travel, so the forward sweep still hides a noise-free scatterer with
    its leading edge: the scatterer depth lies in the leading-edge interval
    of the step that hides it (brute-force occlusion of the forward model),
    that interval's bins get +A, and the first interval runs backwards."""
    geom = S.detector_geometry(3, 2, roi_origin=(30, 0), det_rows=64, det_cols=64)
    fwd = S.wire_path(41)
    wires = np.concatenate([fwd[:1] + 0.4 * (fwd[1] - fwd[0]), fwd])
    e = S.bin_edges(-50, 50, 1.0)
    A = 1000.0
    d = O.depths(geom, wires)
    assert (d[:, :, 1] < d[:, :, 0]).all() and (np.diff(d[:, :, 1:], axis=2) > 0).all()
    for s in (0.0101, 0.0233):
        scat = S.Scatterers(np.array([s]), np.array([A]))
        images = np.rint(S.expected_counts(geom, wires, scat)).astype(np.uint16)
        out = O.reconstruct(geom, wires, images, e)
        for r in range(3):
            vis = images[:, r, 0] > 0
            kstar = int(np.argmin(vis))                 # first hidden step
            assert kstar > 1 and vis[:kstar].all() and not vis[kstar:].any()
            lo, hi = d[r, 0, kstar - 1], d[r, 0, kstar]
            assert lo <= s <= hi
            jlo = int(np.searchsorted(e, lo, "right") - 1)
            jhi = int(np.searchsorted(e, hi, "right") - 1)
            col = out[:, r, 0]
            assert col[jlo:jhi + 1].sum() == pytest.approx(A, abs=1e-9)
            assert np.abs(col).sum() == pytest.approx(A, abs=1e-9)


def test_row_offsets_follow_the_forward_model():
    """Rows asked for by offset (r0, nrows) are those rows of the detector.
    Three rows 5 mm apart along z (their depth sequences about 5 um apart), one
    noise-free scatterer: each row is hidden at the step that the forward
    model's brute-force occlusion gives for that row, its depths asked for
    alone put the scatterer in that step's leading-edge interval, and its
    reconstruction asked for alone puts +A on that interval's bins."""
    geom = S.detector_geometry(3, 1)
    geom["det_origin"] = [0.0, S.DET_Y_MM, -5.0]
    geom["row_step"] = [0.0, 0.0, 5.0]
    wires = S.wire_path(41)
    e = S.bin_edges(-50, 50, 1.0)
    A, s = 1000.0, 0.0201
    images = np.rint(S.expected_counts(geom, wires, S.Scatterers(np.array([s]),
                                                                 np.array([A])))).astype(np.uint16)
    hidden_at = []
    for r in range(3):
        vis = images[:, r, 0] > 0
        kstar = int(np.argmin(vis))                     # first hidden step
        assert kstar > 0 and vis[:kstar].all() and not vis[kstar:].any()
        hidden_at.append(kstar)
        d = O.depths(geom, wires, r0=r, nrows=1)[0, 0]
        lo, hi = d[kstar - 1], d[kstar]
        assert lo <= s <= hi
        col = O.reconstruct(geom, wires, images, e, r0=r, nrows=1)[:, 0, 0]
        jlo = int(np.searchsorted(e, lo, "right") - 1)
        jhi = int(np.searchsorted(e, hi, "right") - 1)
        assert col[jlo:jhi + 1].sum() == pytest.approx(A, abs=1e-9)
        assert np.abs(col).sum() == pytest.approx(A, abs=1e-9)
    assert len(set(hidden_at)) == 3                     # the rows are told apart


def _refused(geom, wires, edges=None, images=None):
    edges = S.bin_edges(-50, 50, 1.0) if edges is None else edges
    if images is None:
        images = np.zeros((len(wires), geom["rows"], geom["cols"]), np.uint16)
    with pytest.raises(O.OracleError) as ei:
        O.reconstruct(geom, wires, images, edges)
    return str(ei.value)


def test_degenerate_geometries_are_refused():
    """Where the method has no answer the oracle refuses rather than guess:
    a beam along the wire axis (no plane to project into), a wire path with
    no travel along the beam (no leading edge), a pixel inside the wire, a
    pixel whose tangent lines meet the beam before the wire (the wire then
    hides nothing on the beam from it), bins that do not increase, fewer
    than two steps."""
    g = S.detector_geometry(2, 2)
    w = S.wire_path(5)
    along = dict(g, beam_dir=[1.0, 0.0, 0.0])
    assert _refused(along, w) == "bad geometry"
    still = w.copy()
    still[:, 2] = still[0, 2]
    still[:, 0] = np.arange(5) * 0.01               # moving along the axis only
    assert _refused(g, still) == "bad geometry"
    inside = S.detector_geometry(1, 1)
    inside["det_origin"] = [0.0, S.WIRE_Y_MM, S.WIRE_Z0_MM + 0.002]
    assert _refused(inside, w) == "bad geometry"
    between = S.detector_geometry(1, 1)
    between["det_origin"] = [0.0, 0.3, 0.0]         # below the wire, above the beam
    assert _refused(between, w) == "bad geometry"
    e = S.bin_edges(-50, 50, 1.0).copy()
    e[7] = e[6]
    assert _refused(g, w, edges=e) == "bad argument"
    assert _refused(g, w[:1]) == "bad argument"
    # and the regular geometry itself is accepted
    O.reconstruct(g, w, np.zeros((5, 2, 2), np.uint16), S.bin_edges(-50, 50, 1.0))
