"""The N > 1 path of bench.py runs independent replicas (the solve does not
shard): the job's throughput is the sum of the replicas' units over the
slowest replica's time.  Checked with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [120.0, 200.0][rank]           # rank 1 is the slowest
    units = [1000, 1000][rank]
    value, ms_max = bench.aggregate_over_ranks(ms, units)
    q.put((rank, value, ms_max))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for _, value, ms_max in res:
        assert ms_max == pytest.approx(200.0)
        assert value == pytest.approx(2000 / 0.2)      # 2000 DOFs in the slowest rank's 200 ms


def test_single_process_aggregation():
    import bench
    v, ms = bench.aggregate_over_ranks(250.0, 500)
    assert ms == 250.0 and v == pytest.approx(2000.0)
