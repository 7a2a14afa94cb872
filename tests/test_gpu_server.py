"""Serving: continuous admission against a memory budget, uploads overlapped
with other requests' kernels; every result must be the same alone and in the
mix, and the same as dr_reconstruct's."""
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


def _requests():
    a = synth.tiny_scan(41, rows=32, cols=256, K=61)
    b = synth.tiny_scan(42, rows=16, cols=128, K=301, n_scat=2)
    b.edges = synth.bin_edges(-100.0, 320.0, 2.0)
    c = synth.tiny_scan(43, rows=8, cols=64, K=25)
    c.edges = synth.bin_edges(-30.0, 60.0, 0.5)
    scans = [a, b, c, a, b, c]
    out = []
    for i, sc in enumerate(scans):
        im = sc.images if i < 3 else synth.tiny_scan(50 + i, rows=sc.geom["rows"],
                                                     cols=sc.geom["cols"], K=sc.K).images
        out.append((sc, torch.from_numpy(np.ascontiguousarray(im).view(np.int16)).pin_memory()))
    return out


def _result(srv, rid, sc):
    dst = torch.empty((sc.B, sc.geom["rows"], sc.geom["cols"]), device="cuda")
    srv.fetch_into(rid, dst)
    torch.cuda.synchronize()
    return dst


def test_same_result_alone_and_in_the_mix():
    reqs = _requests()
    srv = dr.Server(budget_bytes=1 << 30, slots=4)
    alone = []
    for sc, h in reqs:
        rid = srv.submit(sc.geom, sc.wires, sc.edges, h)
        srv.wait(rid, timeout=60)
        alone.append(_result(srv, rid, sc))
        srv.release(rid)
    ids = [srv.submit(sc.geom, sc.wires, sc.edges, h) for sc, h in reqs]
    mixed = []
    for rid, (sc, _) in zip(ids, reqs):
        srv.wait(rid, timeout=60)
        mixed.append(_result(srv, rid, sc))
        _, times = srv.fetch(rid)
        # plans are built ahead of admission by the planner threads
        assert (times["submitted"] <= times["planned"] <= times["admitted"] <= times["issued"]
                <= times["uploaded"] <= times["done"])
        assert 0 < times["copy"] <= times["done"] - times["admitted"]
    for rid in ids:
        srv.release(rid)
    st = srv.stats()
    assert st["completed"] == 12 and st["failed"] == 0 and st["arena_used"] == 0
    assert st["plans_built"] == 3                      # plan cache reused
    for (sc, h), a, m in zip(reqs, alone, mixed):
        assert torch.equal(a.view(torch.int32), m.view(torch.int32))
        plan = dr.Plan(sc.geom, sc.wires, sc.edges)
        ref = plan.reconstruct(h.cuda())
        torch.cuda.synchronize()
        assert torch.equal(ref.view(torch.int32), m.view(torch.int32))
    srv.close()


def test_admission_waits_for_memory_and_rejects_oversize():
    reqs = _requests()
    sc, h = reqs[0]
    need = sc.P * (2 * sc.K + 4 * sc.B)
    # room for one request of this size at a time
    srv = dr.Server(budget_bytes=int(need * 1.5) + (1 << 20), slots=4)
    ids = [srv.submit(sc.geom, sc.wires, sc.edges, h) for _ in range(3)]
    srv.wait(ids[0], timeout=60)
    # the second cannot be admitted until the first output is released
    assert srv.poll(ids[1]) == "queued"
    srv.release(ids[0])
    srv.wait(ids[1], timeout=60)
    srv.release(ids[1])
    srv.wait(ids[2], timeout=60)
    srv.release(ids[2])
    big = synth.tiny_scan(44, rows=64, cols=256, K=61)
    hb = torch.from_numpy(big.images.view(np.int16)).pin_memory()
    rid = srv.submit(big.geom, big.wires, big.edges, hb)
    with pytest.raises(dr.DrError) as ex:
        srv.wait(rid, timeout=60)
    assert ex.value.status == 5
    srv.release(rid)
    assert srv.stats()["arena_used"] == 0
    with pytest.raises(dr.DrError):
        srv.poll(123456)
    srv.close()


def test_served_scans_take_every_kernel():
    """The server builds its plans with dr_plan, so a rotated detector is
    served by the per-pixel kernel and a wire that also climbs across the
    beam by the interval kernel; each result equals dr_reconstruct's."""
    rot = synth.spot_scan(45, 6, 96, 33, 6, -60.0, 60.0, 1.0, rotate_deg=8.0,
                          depth_range=(-0.03, 0.03))
    climb = synth.tiny_scan(46, rows=4, cols=40, K=30, roi_origin=(1900, 1000),
                            det_rows=2048, det_cols=2048)
    climb.wires = synth.wire_path(30, dy=0.005)
    climb.edges = synth.bin_edges(-200.0, -140.0, 1.0)
    srv = dr.Server(budget_bytes=1 << 28, slots=2)
    for sc, kernel in ((rot, "pixels"), (climb, "intervals")):
        plan = dr.Plan(sc.geom, sc.wires, sc.edges)
        assert plan.info()["kernel"] == kernel
        h = torch.from_numpy(np.ascontiguousarray(sc.images).view(np.int16)).pin_memory()
        rid = srv.submit(sc.geom, sc.wires, sc.edges, h)
        srv.wait(rid, timeout=60)
        got = _result(srv, rid, sc)
        srv.release(rid)
        ref = plan.reconstruct(h.cuda())
        torch.cuda.synchronize()
        assert torch.equal(ref.view(torch.int32), got.view(torch.int32))
    srv.close()
