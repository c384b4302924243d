"""The multi-rank leg of bench.py on CPU: two gloo ranks with different step
times report the slowest rank's time and the whole-job throughput (replicas:
every rank does one matvec per step, no collective on the data path)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [2.0, 3.5][rank]
    ms = bench.max_over_ranks(local_ms, world)
    out[rank] = (ms, bench.job_throughput(ms, world))
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_bench():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        ms, value = out[r]
        assert ms == pytest.approx(3.5)
        assert value == pytest.approx(2 * 1000.0 / 3.5)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(1.25, 1) == 1.25
    assert bench.job_throughput(2.0, 1) == pytest.approx(500.0)
