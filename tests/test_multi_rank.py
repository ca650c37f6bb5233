"""The multi-process path of bench.py on CPU: two gloo ranks (one process per GPU in
the real run) report the whole-job throughput over the slowest rank, as the bench's
contract asks (max over ranks, value = ranks x steps / time)."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench._dist_env()
    assert (r, w, local) == (rank, world, rank)
    # rank 1 is the slow one: 300 ms for 10 steps against 200 ms
    value, total = bench._job_throughput(200.0 + 100.0 * rank, 10, world, "cpu")
    out[rank] = (value, total)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_report_max_over_ranks():
    pytest.importorskip("torch.distributed")
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        value, total = out[r]
        assert total == 300.0
        assert abs(value - 2 * 10 / 0.3) < 1e-9
