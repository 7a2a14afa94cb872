"""The reconstruction entry point that allocates nothing (GPU).

dr_reconstruct_rows_static serves callers that cannot call cudaMalloc (their
device memory belongs to another allocator, or their pipeline may not
allocate while running).  It keeps its geometry tables in a fixed device
array inside the library, so its results must match the plan-based entry
point (dr_plan + dr_reconstruct) within the parity tolerance of the other
GPU tests, call after call, even though each call overwrites the array.
This file is collected last so a run that stops at the first failure has
already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2201_13309_gb300 import dr, synth  # noqa: E402

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


def test_static_entry_matches_plan_entry_on_two_calls_in_a_row():
    a = synth.tiny_scan(21)                                  # 64x64, K=41, B=101
    b = synth.tiny_scan(22, rows=24, cols=200, K=77)         # other sizes, ragged tile
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
        _check_close(out.cpu().numpy(), ref.cpu().numpy(), scan.images)
    # the same scan again after the other one overwrote the device tables
    out = torch.empty((a.B, 64, 64), device="cuda")
    dr.reconstruct_rows_static(a.geom, a.wires, a.edges, _dev(a.images), out)
    ref = dr.Plan(a.geom, a.wires, a.edges).reconstruct(_dev(a.images))
    torch.cuda.synchronize()
    _check_close(out.cpu().numpy(), ref.cpu().numpy(), a.images)


def test_static_entry_rejects_what_does_not_fit():
    big = synth.detector_geometry(65000, 8)        # 65000 * 32 B of row tables > 2 MiB
    with pytest.raises(dr.DrError) as ex:
        dr.reconstruct_rows_static(big, synth.wire_path(3000), synth.bin_edges(-50, 50, 1.0),
                                   None, None)
    assert ex.value.status == 5 and "limit" in str(ex.value)
    rot = synth.detector_geometry(8, 8, rotate_deg=10.0)
    with pytest.raises(dr.DrError) as ex:
        dr.reconstruct_rows_static(rot, synth.wire_path(5), synth.bin_edges(-5, 5, 1.0),
                                   None, None)
    assert ex.value.status == 8
