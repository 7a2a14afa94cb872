"""Pixel selection (the paper's pixel-percentage experiment): exact activity,
ordered compaction, and compacted reconstruction equal to the full one."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

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


@pytest.mark.parametrize("rotate", [0.0, 7.0])
def test_selection_sweep(rotate):
    sc = synth.spot_scan(71, 48, 160, 41, 20, -60.0, 60.0, 1.0, rotate_deg=rotate,
                         depth_range=(-0.03, 0.03))
    img = _dev(sc.images)
    act = dr.pixel_activity(img)
    want = np.abs(np.diff(sc.images.astype(np.int64), axis=0)).sum(0)
    assert np.array_equal(act.cpu().numpy().astype(np.int64), want)
    plan = dr.Plan(sc.geom, sc.wires, sc.edges)
    full = plan.reconstruct(img).reshape(sc.B, -1)
    flat = act.reshape(-1)
    for pct in (3, 25, 50, 70, 95, 100):   # lists under 90% walk, denser ones are staged
        thr = float(np.percentile(want, 100 - pct)) if pct < 100 else -1.0
        idx, n = dr.select_pixels(flat, thr)
        ref_idx = np.nonzero(want.reshape(-1) >= thr)[0]
        assert n == ref_idx.size and np.array_equal(idx.cpu().numpy(), ref_idx)
        out = plan.reconstruct_selected(img, idx, n)
        torch.cuda.synchronize()
        assert torch.equal(out.view(torch.int32), full[:, idx.long()].view(torch.int32))


@pytest.mark.parametrize("rows,cols,K", [(3, 64, 7), (5, 37, 7), (2, 8, 2), (4, 40, 402)])
def test_activity_exact(rows, cols, K):
    """Sum |dI| with 16-byte loads (pixel count a multiple of 8) and with the
    2-pixel form (odd count), step counts with and without a tail of the
    4-step unroll, extreme values (0 / 65535 alternating): the exact integer
    sum rounded once to FP32 (exact below 2^24; the extreme pixels of the
    402-step stack sum to 26.3 M)."""
    rng = np.random.Generator(np.random.PCG64(rows * cols + K))
    im = rng.integers(0, 65536, (K, rows, cols), dtype=np.uint16)
    im[::2, 0, :4] = 0
    im[1::2, 0, :4] = 65535
    act = dr.pixel_activity(_dev(im)).cpu().numpy()
    want = np.abs(np.diff(im.astype(np.int64), axis=0)).sum(0)
    assert np.array_equal(act, want.astype(np.float32))


def test_selection_edge_cases():
    sc = synth.tiny_scan(72, rows=4, cols=64, K=9)
    img = _dev(sc.images)
    act = dr.pixel_activity(img).reshape(-1)
    idx, n = dr.select_pixels(act, 1e30)
    assert n == 0
    plan = dr.Plan(sc.geom, sc.wires, sc.edges)
    out = plan.reconstruct_selected(img, idx, 0, out=torch.empty((sc.B, 1), device="cuda"))
    big = torch.rand(3 * 4096 + 17, device="cuda")       # several chunks, ragged tail
    idx, n = dr.select_pixels(big, 0.5)
    ref = torch.nonzero(big >= 0.5).reshape(-1).int()
    assert n == ref.numel() and torch.equal(idx, ref)
