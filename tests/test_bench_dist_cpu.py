"""bench.py's multi-process path on CPU: two gloo ranks, max-over-ranks
timing and the whole-job rate; the reference arm's non-zero ranks exit
without work."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench

    tdist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 100.0 + 50.0 * rank          # rank 1 is the slowest
    mx = bench.reduce_max(local_ms, torch.device("cpu"))
    rate = bench.whole_job_rate(1000, 10, world, mx)
    w, r, lr = bench.dist_setup()
    tdist.barrier()
    tdist.destroy_process_group()
    q.put((rank, mx, rate, w, r, lr))


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, rate, w, r, lr in out:
        assert mx == 150.0 and w == 2 and r == rank == lr
        assert rate == pytest.approx(2 * 1000 * 10 / 0.150)


def test_single_process_reduce_is_identity():
    import bench

    assert bench.reduce_max(12.5, torch.device("cpu")) == 12.5
    assert bench.whole_job_rate(4, 5, 1, 2000.0) == pytest.approx(10.0)


def test_reference_arm_other_ranks_do_no_work():
    import argparse

    import bench

    args = argparse.Namespace(steps=3, warmup=3)
    assert bench.run_reference(args, 2, 1) == 0


def test_batch_wave_packing():
    import bench
    from tests.gen import synth

    specs = [synth.batch_scan_spec(s) for s in range(64)]
    waves = bench.batch_waves(specs, 120e9)
    assert sum(len(w) for w in waves) == 64
    for w in waves:
        need = sum(sp.P * (2 * sp.K + 4 * sp.B) for sp in w)
        assert need <= 120e9 or len(w) == 1
