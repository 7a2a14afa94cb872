"""The bounded-wait failure path on the GPU, without a fault: a kernel whose
barrier nothing completes gives up after its time limit, records the
timeout code for the host, and the context stays usable (a reconstruction
right after it matches the oracle)."""
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


def test_bounded_wait_runs_out_and_context_stays_usable():
    st, word = dr.selftest_wait_timeout(20.0)
    assert st == 7 and word == 1                      # DR_ERR_TIMEOUT, kDevTmaTimeout
    assert "ran out" in dr.lib().dr_last_error().decode()
    sc = synth.tiny_scan(93, rows=8, cols=32, K=17)
    plan = dr.Plan(sc.geom, sc.wires, sc.edges)
    out = plan.reconstruct(torch.from_numpy(sc.images.view(np.int16)).cuda())
    torch.cuda.synchronize()
    plan.check_device()
    ref = O.reconstruct(sc.geom, sc.wires, sc.images, sc.edges)
    s = np.abs(np.diff(sc.images.astype(np.int64), axis=0)).sum(0)[None]
    assert np.all(np.abs(out.cpu().numpy() - ref) <= 1e-4 * s)


def test_bounded_wait_bad_arguments():
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    L = dr.lib()
    import ctypes
    assert L.dr_selftest_wait_timeout(ctypes.c_void_p(status.data_ptr()), 0.0, None) == 1
    assert L.dr_selftest_wait_timeout(ctypes.c_void_p(status.data_ptr()), 5000.0, None) == 1
    assert L.dr_selftest_wait_timeout(None, 10.0, None) == 1
