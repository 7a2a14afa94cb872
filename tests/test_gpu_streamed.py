"""Out-of-core streamed form (row slabs through a small workspace, uploads,
kernels and downloads overlapped): bitwise equal to the in-core result."""
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


def _case(sc, slab_rows, ws_slabs=3, **kw):
    plan = dr.Plan(sc.geom, sc.wires, sc.edges, **kw)
    h_img = torch.from_numpy(np.ascontiguousarray(sc.images).view(np.int16)).pin_memory()
    ref = plan.reconstruct(h_img.cuda())
    h_out = torch.full((sc.B, sc.geom["rows"], sc.geom["cols"]), float("nan"),
                       dtype=plan.out_torch_dtype()).pin_memory()
    W, K, B = sc.geom["cols"], sc.K, sc.B
    osz = 2 if kw.get("out_dtype") == "bf16" else 4
    per = -(-slab_rows * W * K * 2 // 256) * 256 + -(-slab_rows * W * B * osz // 256) * 256
    ws = torch.empty(per * ws_slabs, dtype=torch.uint8, device="cuda")
    plan.reconstruct_streamed(h_img, h_out, ws, slab_rows=slab_rows)
    torch.cuda.synchronize()
    return ref.cpu(), h_out


@pytest.mark.parametrize("slab_rows", [1, 5, 16, 64])
def test_streamed_equals_in_core(slab_rows):
    sc = synth.tiny_scan(61, rows=37, cols=256, K=61)
    ref, got = _case(sc, slab_rows)
    assert torch.equal(ref.view(torch.int32), got.view(torch.int32))


def test_streamed_per_pixel_geometry_and_bf16():
    sc = synth.spot_scan(62, 21, 96, 33, 6, -60.0, 60.0, 1.0, rotate_deg=8.0,
                         depth_range=(-0.03, 0.03))
    ref, got = _case(sc, 4)
    assert torch.equal(ref.view(torch.int32), got.view(torch.int32))
    sc2 = synth.tiny_scan(63, rows=19, cols=64, K=41)
    ref, got = _case(sc2, 3, out_dtype="bf16")
    assert torch.equal(ref.view(torch.int16), got.view(torch.int16))


def test_streamed_rejects_small_workspace():
    sc = synth.tiny_scan(64, rows=8, cols=64, K=21)
    plan = dr.Plan(sc.geom, sc.wires, sc.edges)
    h_img = torch.from_numpy(sc.images.view(np.int16)).pin_memory()
    h_out = torch.empty((sc.B, 8, 64)).pin_memory()
    ws = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(dr.DrError) as ex:
        plan.reconstruct_streamed(h_img, h_out, ws, slab_rows=4)
    assert ex.value.status == 5


def test_streamed_download_path():
    """A pageable host output (not mapped into the device's address space)
    and a plan of two runs (a path that turns back) take the download stage
    instead of the kernels writing to the host: bitwise the in-core result."""
    sc = synth.tiny_scan(65, rows=13, cols=64, K=31)
    plan = dr.Plan(sc.geom, sc.wires, sc.edges)
    h_img = torch.from_numpy(np.ascontiguousarray(sc.images).view(np.int16)).pin_memory()
    ref = plan.reconstruct(h_img.cuda()).cpu()
    h_out = torch.full(tuple(ref.shape), float("nan"))  # pageable
    ws = torch.empty(16 << 20, dtype=torch.uint8, device="cuda")
    plan.reconstruct_streamed(h_img, h_out, ws, slab_rows=4)
    torch.cuda.synchronize()
    assert torch.equal(ref.view(torch.int32), h_out.view(torch.int32))
    a = synth.wire_path(16)
    b = synth.wire_path(11, z0=a[-1, 2], dz=-0.001)[1:]
    wires = np.concatenate([a, b])
    back = synth.Scan(sc.geom, wires, sc.edges, sc.images[:26])
    plan2 = dr.Plan(back.geom, back.wires, back.edges)
    assert plan2.info()["parts"] == 2
    h_img2 = torch.from_numpy(np.ascontiguousarray(back.images).view(np.int16)).pin_memory()
    ref2 = plan2.reconstruct(h_img2.cuda()).cpu()
    h_out2 = torch.full(tuple(ref2.shape), float("nan")).pin_memory()
    plan2.reconstruct_streamed(h_img2, h_out2, ws, slab_rows=5)
    torch.cuda.synchronize()
    assert torch.equal(ref2.view(torch.int32), h_out2.view(torch.int32))


def test_streamed_plain_loads_and_ragged_slab():
    """A width whose rows are not 16-byte multiples (plain loads, so the
    download path even with a pinned output) and a last slab shorter than
    the others: bitwise the in-core result."""
    sc = synth.tiny_scan(66, rows=11, cols=70, K=23)
    ref, got = _case(sc, 4)
    assert torch.equal(ref.view(torch.int32), got.view(torch.int32))
