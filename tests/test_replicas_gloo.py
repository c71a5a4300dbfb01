"""CPU test of the multi-rank path of bench.py: N replicas of the hot path,
one per GPU, whose job time is the slowest rank's and whose throughput is
the columns of all ranks over that time.  Two gloo ranks stand in for two
GPUs; no collective is on the data path, only the timing reduction."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, ms_by_rank, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms = bench.max_over_ranks(ms_by_rank[rank], dist, "cpu")
        out[rank] = (ms, bench.replica_value(2048, world, ms))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ms_by_rank", [(600.0, 700.0), (812.5, 640.25)])
def test_two_ranks_report_the_slowest_rank_and_all_columns(ms_by_rank):
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, world, port, ms_by_rank, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        codes = [p.exitcode for p in procs]
        res = dict(out)
    assert codes == [0, 0], codes
    slow = max(ms_by_rank)
    for r in range(world):
        ms, value = res[r]
        assert ms == slow
        assert value == pytest.approx(2048 * world / (slow / 1e3), rel=1e-15)


def test_one_rank_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(677.25) == 677.25
    assert bench.replica_value(2048, 1, 677.25) == pytest.approx(2048 / 0.67725, rel=1e-15)
