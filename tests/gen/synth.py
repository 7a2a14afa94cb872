"""Seeded synthetic wire-scan inputs (the forward model).

This module produces the inputs that both the CUDA path and the FP64 oracle
consume: detector/wire/beam geometry, the wire path, the depth-bin edges and
the uint16 image stacks of a differential-aperture (wire) scan.  It contains
no reconstruction arithmetic (no tangent depths, no differencing, no
apportioning).  Its only geometry is the physical forward model: a point
scatterer on the incident beam is hidden at a wire step when the straight
segment from the scatterer to the pixel centre passes closer than the wire
radius to the wire axis (brute-force point-to-segment distance in the plane
perpendicular to the axis).

The paper measures on real HDF5 scans from the 34-ID-E beamline (Sec. IV);
those data are not available, so scans shaped like them stand in:

* tiny:  64x64 pixels, 41 steps, 5 scatterers lighting every pixel,
         101 bins of 1 um over [-50, 50] um (bin centres).
* full:  2048x2048 pixels, 401 steps, 200 scatterers each lighting a 5x5
         Gaussian spot, Poisson background of mean 20, 1001 bins over
         [-500, 500] um.
* batch: ROI in {256^2, 512^2, 1024^2, 2048x1024, 2048^2} placed on the
         2048^2 detector, 51..801 steps, bins of 0.5/1/2 um over +-400 um.

Lengths are millimetres in the lab frame.  Beam along +z through the origin,
wire axis along x at y = 0.5 mm, wire centre z_k = -20 um + k * 1 um, flat
detector in the plane y = 510 mm with 0.2 mm pitch centred over the origin;
detector columns run along x (the wire axis) and rows along z.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

PITCH_MM = 0.2
DET_Y_MM = 510.0
WIRE_Y_MM = 0.5
WIRE_R_MM = 0.026
WIRE_Z0_MM = -0.020
WIRE_DZ_MM = 0.001
FULL_DET = 2048


def detector_geometry(rows, cols, roi_origin=(None, None), det_rows=None,
                      det_cols=None, rotate_deg=0.0, tilt_deg=0.0):
    """Geometry dict for an ROI of a flat detector at y = 510 mm.

    ``roi_origin`` is the (row, col) of the ROI's first pixel on a detector of
    ``det_rows x det_cols`` pixels centred over the origin (default: the ROI
    is the whole detector).  ``rotate_deg`` turns the detector in its own
    plane (columns then no longer run along the wire axis, so every pixel has
    its own depth sequence); ``tilt_deg`` tilts the detector about x (rows
    then also move in y).
    """
    det_rows = rows if det_rows is None else det_rows
    det_cols = cols if det_cols is None else det_cols
    r0 = 0 if roi_origin[0] is None else roi_origin[0]
    c0 = 0 if roi_origin[1] is None else roi_origin[1]
    th = math.radians(rotate_deg)
    tl = math.radians(tilt_deg)
    # unit vectors of the detector axes before rotation: col -> x, row -> z
    col_u = np.array([math.cos(th), 0.0, math.sin(th)])
    row_u = np.array([-math.sin(th), 0.0, math.cos(th)])
    # tilt about x: z-components pick up a y-component
    def tilt(v):
        return np.array([v[0], v[2] * math.sin(tl), v[2] * math.cos(tl)])
    col_u, row_u = tilt(col_u), tilt(row_u)
    centre = np.array([0.0, DET_Y_MM, 0.0])
    dr = (r0 - (det_rows - 1) / 2.0) * PITCH_MM
    dc = (c0 - (det_cols - 1) / 2.0) * PITCH_MM
    origin = centre + dr * row_u + dc * col_u
    return {
        "beam_origin": [0.0, 0.0, 0.0],
        "beam_dir": [0.0, 0.0, 1.0],
        "det_origin": origin.tolist(),
        "row_step": (PITCH_MM * row_u).tolist(),
        "col_step": (PITCH_MM * col_u).tolist(),
        "rows": int(rows),
        "cols": int(cols),
        "wire_axis": [1.0, 0.0, 0.0],
        "wire_radius": WIRE_R_MM,
    }


def wire_path(K, z0=WIRE_Z0_MM, dz=WIRE_DZ_MM, y=WIRE_Y_MM, dy=0.0):
    """[K, 3] wire-centre positions: x = 0, y = y + k*dy, z = z0 + k*dz."""
    k = np.arange(K, dtype=np.float64)
    c = np.zeros((K, 3), dtype=np.float64)
    c[:, 1] = y + k * dy
    c[:, 2] = z0 + k * dz
    return c


def bin_edges(lo_um, hi_um, width_um):
    """Edges of bins whose CENTRES run from lo to hi in steps of width (mm).

    "1 um bins over [-50, 50] um (101 bins)" names the bin centres, so the
    edges run from -50.5 to 50.5 um.
    """
    n = int(round((hi_um - lo_um) / width_um)) + 1
    j = np.arange(n + 1, dtype=np.float64)
    return (lo_um - width_um / 2.0 + j * width_um) * 1e-3


def pixel_centres(geom):
    """[rows, cols, 3] lab coordinates of the pixel centres."""
    r = np.arange(geom["rows"], dtype=np.float64)[:, None, None]
    c = np.arange(geom["cols"], dtype=np.float64)[None, :, None]
    return (np.asarray(geom["det_origin"])[None, None, :]
            + r * np.asarray(geom["row_step"])[None, None, :]
            + c * np.asarray(geom["col_step"])[None, None, :])


def hidden_by_wire(source, pixels, centre, axis, radius):
    """True where the segment source->pixel passes within ``radius`` of the
    wire axis (the infinite line through ``centre`` along ``axis``).

    Brute force: project onto the plane perpendicular to the axis and take
    the distance from the projected centre to the projected segment.
    ``pixels`` has shape [..., 3]; the result has shape [...].
    """
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    s = np.asarray(source, dtype=np.float64)
    c = np.asarray(centre, dtype=np.float64)

    def proj(v):
        return v - np.sum(v * a, axis=-1, keepdims=True) * a

    seg = proj(pixels - s)                 # segment direction, from source
    rel = proj(c - s)                      # wire centre relative to source
    den = np.sum(seg * seg, axis=-1)
    t = np.clip(np.sum(rel * seg, axis=-1) / den, 0.0, 1.0)
    closest = t[..., None] * seg - rel
    return np.sqrt(np.sum(closest * closest, axis=-1)) < radius


@dataclass
class Scatterers:
    depth: np.ndarray          # [n] mm along the beam
    peak: np.ndarray           # [n] counts
    spot_row: np.ndarray = field(default=None)  # [n] spot centre row (None: all pixels)
    spot_col: np.ndarray = field(default=None)


def tiny_scatterers(rng, n=5):
    depth = rng.uniform(-0.015, 0.015, n)
    peak = rng.uniform(500.0, 5000.0, n)
    return Scatterers(depth, peak)


def spot_scatterers(rng, n, rows, cols, depth_lo=-0.150, depth_hi=0.150):
    depth = rng.uniform(depth_lo, depth_hi, n)
    peak = np.exp(rng.uniform(math.log(1e2), math.log(6e4), n))
    sr = rng.integers(2, max(rows - 2, 3), n)
    sc = rng.integers(2, max(cols - 2, 3), n)
    return Scatterers(depth, peak, sr, sc)


def expected_counts(geom, wires, scat, background=0.0, spot_sigma=1.0):
    """Noise-free expected counts [K, rows, cols] (float64)."""
    H, W, K = geom["rows"], geom["cols"], wires.shape[0]
    beam_o = np.asarray(geom["beam_origin"], dtype=np.float64)
    beam_d = np.asarray(geom["beam_dir"], dtype=np.float64)
    beam_d = beam_d / np.linalg.norm(beam_d)
    rate = np.full((K, H, W), float(background))
    q = pixel_centres(geom)
    for i in range(scat.depth.shape[0]):
        src = beam_o + scat.depth[i] * beam_d
        if scat.spot_row is None:
            rr, cc = slice(0, H), slice(0, W)
            prof = np.ones((H, W))
        else:
            r0 = max(int(scat.spot_row[i]) - 2, 0)
            c0 = max(int(scat.spot_col[i]) - 2, 0)
            r1 = min(int(scat.spot_row[i]) + 3, H)
            c1 = min(int(scat.spot_col[i]) + 3, W)
            rr, cc = slice(r0, r1), slice(c0, c1)
            dr = np.arange(r0, r1)[:, None] - scat.spot_row[i]
            dc = np.arange(c0, c1)[None, :] - scat.spot_col[i]
            prof = np.exp(-(dr * dr + dc * dc) / (2.0 * spot_sigma ** 2))
        qs = q[rr, cc]
        for k in range(K):
            vis = ~hidden_by_wire(src, qs, wires[k], geom["wire_axis"],
                                  geom["wire_radius"])
            rate[k, rr, cc] += scat.peak[i] * prof * vis
    return rate


def poisson_u16(rng, rate):
    """Poisson draw of ``rate`` clamped to the uint16 range."""
    return np.minimum(rng.poisson(rate), 65535).astype(np.uint16)


@dataclass
class Scan:
    geom: dict
    wires: np.ndarray          # [K, 3]
    edges: np.ndarray          # [B + 1]
    images: np.ndarray = None  # [K, rows, cols] uint16 (None when on device)
    scat: Scatterers = None
    name: str = ""

    @property
    def K(self):
        return int(self.wires.shape[0])

    @property
    def B(self):
        return int(self.edges.shape[0] - 1)

    @property
    def P(self):
        return int(self.geom["rows"] * self.geom["cols"])


def tiny_scan(seed=0, noise=True, rows=64, cols=64, K=41, n_scat=5, **geo_kw):
    """The 64x64, 41-step, 101-bin scan (5 scatterers lighting every pixel)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    geom = detector_geometry(rows, cols, **geo_kw)
    wires = wire_path(K)
    scat = tiny_scatterers(rng, n_scat)
    rate = expected_counts(geom, wires, scat)
    images = poisson_u16(rng, rate) if noise else np.rint(rate).astype(np.uint16)
    return Scan(geom, wires, bin_edges(-50.0, 50.0, 1.0), images, scat, "tiny")


def spot_scan(seed, rows, cols, K, n_scat, lo_um, hi_um, width_um,
              roi_origin=(None, None), det_rows=None, det_cols=None,
              background=20.0, depth_range=(-0.150, 0.150), noise=True,
              **geo_kw):
    """Spot scan generated on the host (small sizes: tests)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    geom = detector_geometry(rows, cols, roi_origin, det_rows, det_cols, **geo_kw)
    wires = wire_path(K)
    scat = spot_scatterers(rng, n_scat, rows, cols, *depth_range)
    rate = expected_counts(geom, wires, scat, background)
    images = poisson_u16(rng, rate) if noise else np.rint(rate).astype(np.uint16)
    return Scan(geom, wires, bin_edges(lo_um, hi_um, width_um), images, scat,
                f"spot{rows}x{cols}")


def spot_contributions(geom, wires, scat, spot_sigma=1.0):
    """Sparse noise-free scatterer contributions for spot scans.

    Returns (flat_index int64 [n], value float32 [n]) into a [K, rows, cols]
    array.  Used to build large scans on a device without a dense host rate.
    """
    H, W, K = geom["rows"], geom["cols"], wires.shape[0]
    beam_o = np.asarray(geom["beam_origin"], dtype=np.float64)
    beam_d = np.asarray(geom["beam_dir"], dtype=np.float64)
    beam_d = beam_d / np.linalg.norm(beam_d)
    idx, val = [], []
    kk = np.arange(K)
    for i in range(scat.depth.shape[0]):
        src = beam_o + scat.depth[i] * beam_d
        r0 = max(int(scat.spot_row[i]) - 2, 0)
        c0 = max(int(scat.spot_col[i]) - 2, 0)
        r1 = min(int(scat.spot_row[i]) + 3, H)
        c1 = min(int(scat.spot_col[i]) + 3, W)
        rs = np.arange(r0, r1)
        cs = np.arange(c0, c1)
        dr = rs[:, None] - scat.spot_row[i]
        dc = cs[None, :] - scat.spot_col[i]
        prof = np.exp(-(dr * dr + dc * dc) / (2.0 * spot_sigma ** 2))
        q = (np.asarray(geom["det_origin"])
             + rs[:, None, None] * np.asarray(geom["row_step"])
             + cs[None, :, None] * np.asarray(geom["col_step"]))
        # [K, nr, nc]: every wire step at once
        vis = ~hidden_by_wire(src, q[None], wires[:, None, None, :], geom["wire_axis"],
                              geom["wire_radius"])
        v = scat.peak[i] * prof[None] * vis
        flat = (kk[:, None, None] * H + rs[None, :, None]) * W + cs[None, None, :]
        idx.append(flat.reshape(-1))
        val.append(v.reshape(-1))
    if not idx:
        return np.zeros(0, np.int64), np.zeros(0, np.float32)
    return (np.concatenate(idx).astype(np.int64),
            np.concatenate(val).astype(np.float32))


def device_spot_images(geom, wires, scat, seed, background, device,
                       step_chunk=64):
    """Poisson spot-scan image stack built on a CUDA device.

    Returns a torch int16 tensor [K, rows, cols] holding the uint16 bit
    patterns (torch's uint16 support differs between versions).  The noise is
    drawn with a seeded torch generator on the device, one chunk of steps at a
    time, so that multi-GB scans never need a dense host copy.
    """
    import torch

    H, W, K = geom["rows"], geom["cols"], wires.shape[0]
    idx, val = spot_contributions(geom, wires, scat)
    idx_t = torch.from_numpy(idx).to(device)
    val_t = torch.from_numpy(val).to(device)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    out = torch.empty((K, H, W), dtype=torch.int16, device=device)
    plane = H * W
    for k0 in range(0, K, step_chunk):
        k1 = min(K, k0 + step_chunk)
        rate = torch.full(((k1 - k0) * plane,), float(background),
                          dtype=torch.float32, device=device)
        sel = (idx_t >= k0 * plane) & (idx_t < k1 * plane)
        rate.index_add_(0, idx_t[sel] - k0 * plane, val_t[sel])
        counts = torch.poisson(rate, generator=gen).clamp_(0, 65535)
        out[k0:k1] = counts.to(torch.int32).to(torch.int16).view(k1 - k0, H, W)
        del rate, counts
    return out


def full_scan_spec(seed=0):
    """2048x2048 pixels, 401 steps, 1001 bins of 1 um over [-500, 500] um."""
    rng = np.random.Generator(np.random.PCG64(seed))
    geom = detector_geometry(FULL_DET, FULL_DET)
    wires = wire_path(401)
    scat = spot_scatterers(rng, 200, FULL_DET, FULL_DET)
    return Scan(geom, wires, bin_edges(-500.0, 500.0, 1.0), None, scat, "full")


ROI_CHOICES = ((256, 256), (512, 512), (1024, 1024), (2048, 1024), (2048, 2048))
BIN_WIDTHS_UM = (0.5, 1.0, 2.0)


def batch_scan_spec(seed, rotate_deg=0.0):
    """One scan of the uneven batch: ROI, step count and bin width drawn from
    the seeded distribution; scatterer count 200 * area / 2048^2 (min 5).
    rotate_deg turns the detector in its plane (every pixel then has its own
    depth sequence)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    rows, cols = ROI_CHOICES[int(rng.integers(0, len(ROI_CHOICES)))]
    K = int(rng.integers(51, 802))
    width = BIN_WIDTHS_UM[int(rng.integers(0, len(BIN_WIDTHS_UM)))]
    r0 = int(rng.integers(0, FULL_DET - rows + 1))
    c0 = int(rng.integers(0, FULL_DET - cols + 1))
    n_scat = max(5, int(round(200 * rows * cols / FULL_DET ** 2)))
    geom = detector_geometry(rows, cols, (r0, c0), FULL_DET, FULL_DET, rotate_deg=rotate_deg)
    wires = wire_path(K)
    scat = spot_scatterers(rng, n_scat, rows, cols)
    return Scan(geom, wires, bin_edges(-400.0, 400.0, width), None, scat,
                f"batch{seed}")
