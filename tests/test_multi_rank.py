"""The replicated multi-GPU path of bench.py, host side only: each rank runs an
independent copy of the workload (no data-path collective); the whole-job
figures are the slowest rank's time and the sum of all ranks' work. Checked with
two gloo ranks on the CPU."""
import os

import pytest
import torch.multiprocessing as mp


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, counts = bench.reduce_over_ranks(dist, 100.0 + 50.0 * rank, [80 + rank, 21000 + 10 * rank], "cpu")
        out.put((rank, ms, counts))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_max_time_and_summed_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, counts in res:
        assert ms == 150.0                      # the slowest rank
        assert counts == [161, 42010]           # all ranks' solves and matvecs
