"""Seeded random scans through dr_plan + dr_reconstruct against the FP64
oracle (GPU): wire paths of every kind the plan distinguishes (straight
either way, turning back along the beam, climbing across the beam with
jitter, repeated positions, steps too fine for the FP32 grid), aligned,
rotated and tilted detectors, even and uneven bins, leading, trailing and
both edges.  Whatever kernel the plan picks, every FP32 bin must be within
1e-4 of its pixel's sum |dI| of the oracle, and bins of pixels with no
change must be exactly zero."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2201_13309_gb300 import dr  # noqa: E402
from tests.gen import synth  # noqa: E402

pytestmark = pytest.mark.gpu

PATHS = ("forward", "backward", "turn", "climb", "repeat", "fine")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()


def random_scan(seed):
    rng = np.random.Generator(np.random.PCG64(1000 + seed))
    rows = int(rng.integers(1, 9))
    cols = int(rng.choice([8, 24, 40, 64, 70, 96]))
    K = int(rng.integers(6, 48))
    kind = PATHS[seed % len(PATHS)]
    geom = synth.detector_geometry(rows, cols, roi_origin=(int(rng.integers(0, 2040)),
                                                           int(rng.integers(0, 1900))),
                                   det_rows=2048, det_cols=2048,
                                   rotate_deg=float(rng.choice([0.0, 0.0, 7.0, -12.0])),
                                   tilt_deg=float(rng.choice([0.0, 0.0, 4.0])))
    dz = float(rng.uniform(0.5e-3, 2e-3))
    wires = synth.wire_path(K, dz=dz)
    if kind == "backward":
        wires = wires[::-1].copy()
    elif kind == "turn":
        m = int(rng.integers(2, K - 2))
        wires[m:, 2] = wires[m, 2] - (wires[m:, 2] - wires[m, 2]) * 0.7
    elif kind == "climb":
        wires[:, 1] += np.arange(K) * 0.0035 + rng.normal(0.0, 0.0004, K)
    elif kind == "repeat":
        m = int(rng.integers(1, K - 1))
        wires[m] = wires[m - 1]
    elif kind == "fine":
        m = int(rng.integers(1, K - 1))
        wires[m:, 2] -= dz - 1e-9
    d = np.concatenate([O.depths(geom, wires, "leading"), O.depths(geom, wires, "trailing")])
    lo, hi = d.min() * 1e3, d.max() * 1e3  # both edges' depths (um)
    scat = synth.Scatterers(rng.uniform(d.min(), d.max(), 4), rng.uniform(300.0, 5000.0, 4))
    images = synth.poisson_u16(rng, synth.expected_counts(geom, wires, scat, background=25.0))
    if rng.random() < 0.5:
        edges = synth.bin_edges(np.floor(lo) - 3, np.ceil(hi) + 3,
                                float(rng.choice([0.25, 0.5, 1.0, 2.0])))
    else:  # uneven bins, some wider than the depth steps, some narrower
        n = int(rng.integers(8, 80))
        edges = np.sort(rng.uniform(lo - 5.0, hi + 5.0, n + 1)) * 1e-3
        edges = np.unique(edges)
    edge = str(rng.choice(["leading", "trailing", "both"]))
    return synth.Scan(geom, wires, edges, images), edge, kind


@pytest.mark.parametrize("seed", range(48))
def test_random_scan_against_oracle(seed):
    sc, edge, kind = random_scan(seed)
    try:
        plan = dr.Plan(sc.geom, sc.wires, sc.edges, edge=edge)
    except dr.DrError as e:
        # the one refusal a random path can meet: a wire that ends where it
        # started along the beam (no travel) for both edges
        assert e.status == 2, (kind, edge, str(e))
        return
    img = torch.from_numpy(np.ascontiguousarray(sc.images).view(np.int16)).cuda()
    out = plan.reconstruct(img)
    torch.cuda.synchronize()
    plan.check_device()
    got = out.cpu().numpy().astype(np.float64)
    want = O.reconstruct(sc.geom, sc.wires, sc.images, sc.edges, edge)
    s = np.abs(np.diff(sc.images.astype(np.int64), axis=0)).sum(0)[None]
    err = np.abs(got - want)
    info = plan.info()
    assert np.all(err <= 1e-4 * s), (kind, edge, info["kernel"],
                                     float((err / np.maximum(s, 1)).max()))
    assert np.all(got[np.broadcast_to(s == 0, got.shape)] == 0)


def test_random_scans_batched_and_streamed():
    """The random scans whose plans a batch takes (single run, single edge,
    widths a multiple of 8) in one batch, bitwise their per-scan launches;
    every random scan streamed through two-row slabs into a pinned host
    output, bitwise its in-core result."""
    jobs, refs, keep = [], [], []
    ws = torch.empty(32 << 20, dtype=torch.uint8, device="cuda")
    for seed in range(24):
        sc, edge, kind = random_scan(seed)
        try:
            plan = dr.Plan(sc.geom, sc.wires, sc.edges, edge=edge)
        except dr.DrError:
            continue
        h_img = torch.from_numpy(np.ascontiguousarray(sc.images).view(np.int16)).pin_memory()
        img = h_img.cuda()
        ref = plan.reconstruct(img)
        h_out = torch.full(tuple(ref.shape), float("nan")).pin_memory()
        plan.reconstruct_streamed(h_img, h_out, ws, slab_rows=2)
        torch.cuda.synchronize()
        assert torch.equal(h_out.view(torch.int32), ref.cpu().view(torch.int32)), (seed, kind)
        info = plan.info()
        if info["parts"] == 1 and sc.geom["cols"] % 8 == 0:
            jobs.append((plan, img, torch.full_like(ref, float("nan"))))
            refs.append(ref)
            keep.append(plan)
    assert len(jobs) >= 8
    kinds = {p.info()["kernel"] for p in keep}
    assert {"rows", "intervals"} <= kinds
    dr.batch_reconstruct(jobs)
    for (_, _, out), ref in zip(jobs, refs):
        assert torch.equal(out.view(torch.int32), ref.view(torch.int32))
