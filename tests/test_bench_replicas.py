"""The multi-GPU path of the benchmark is replicas only (no exchange step):
each rank times its own copy of the step, the slowest rank's time counts,
and the whole-job rate sums every rank's units. The rank aggregation runs
here on CPU with two gloo processes."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as d
    d.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    try:
        # rank r took 1 + r seconds for the device-timed steps and 5 - r end to end
        t, e = bench.max_over_ranks(d, [1.0 + rank, 5.0 - rank], "cpu")
        out[rank] = (t, e, bench.whole_job_rate(300 * 10, world, t))
    finally:
        d.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_replica():
    if not dist.is_available():
        pytest.skip("torch.distributed unavailable")
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        t, e, rate = res[rank]
        assert (t, e) == (2.0, 5.0)
        assert rate == pytest.approx(300 * 10 * 2 / 2.0)


def test_single_process_keeps_its_own_times():
    import bench
    assert bench.max_over_ranks(None, [3.0, 4.0], "cpu") == [3.0, 4.0]
    assert bench.whole_job_rate(3000, 1, 2.0) == 1500.0
