"""The multi-rank arithmetic of bench.py (`--gpus N` under torchrun) on CPU
with the gloo backend, world size 2: the job's time is the slowest rank's,
its rate the units of all ranks over that time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [12.5, 20.0][rank]                  # rank 1 is the slower one
    ms_max = bench.max_over_ranks(local_ms, dist, "cpu")
    rate = bench.job_rate(world, 1000 * 4, ms_max * 1e-3)
    out.put((rank, ms_max, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, ms_max, rate in res:
        assert ms_max == 20.0                      # both ranks see the slowest time
        assert rate == pytest.approx(2 * 4000 / 0.020)


def test_single_rank_is_the_local_value():
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.job_rate(1, 10, 2.0) == 5.0
