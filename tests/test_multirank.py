"""The N > 1 path of bench.py (replicas, one per rank) on CPU with the gloo
backend: the whole-job value takes the slowest rank's time and every rank's
units, and the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist        # noqa: E402
import torch.multiprocessing as mp      # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t_local = 100.0 + 50.0 * rank                  # ms: rank 1 is the slow one
        t, value = bench.whole_job(t_local, 1000, world)
        out[rank] = (t, value)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_whole_job_takes_the_slowest_rank_and_all_units():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        t, value = res[r]
        assert t == 150.0
        assert value == pytest.approx(world * 1000 / 0.150)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    """A rank other than 0 returns before building any input."""
    sys.path.insert(0, ROOT)
    import bench
    called = []

    def no_inputs(*args, **kwargs):
        called.append(1)
        raise RuntimeError("rank 1 must not build inputs")

    monkeypatch.setattr(bench, "make_inputs", no_inputs)
    monkeypatch.setenv("RANK", "1")

    class Args:
        ntri, extra, steps, warmup = 64, 10, 1, 0

    assert bench.run_reference(Args()) is None
    assert called == []
