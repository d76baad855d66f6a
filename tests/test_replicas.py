"""Multi-GPU is replicas only (the path does not shard): N independent solves,
one per rank.  The host logic of bench.py's N > 1 run -- the job time is the
slowest rank's, the whole-job value counts every rank's work, and the
reference arm prints from rank 0 only -- checked with world_size-2 gloo
process groups on the CPU."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 10.0 + 5.0 * rank          # rank 1 is the slower replica
    ms = bench.max_over_ranks(local_ms, dist)
    out[rank] = (ms, bench.replica_value(world, 1e9, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
    import torch.multiprocessing as mp
    torch = pytest.importorskip("torch")
    port = 29000 + (os.getpid() % 2000)
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    # both ranks see the slowest rank's time; the value counts both ranks' bytes
    assert out[0][0] == out[1][0] == 15.0
    assert out[0][1] == pytest.approx(2 * 1e9 / 15e-3 / 1e9)


def test_single_rank_and_reference_arm_off_rank_zero(capsys):
    import bench
    assert bench.max_over_ranks(3.5, None) == 3.5
    assert bench.replica_value(1, 2e9, 1000.0) == pytest.approx(2.0)

    class Args:
        gpus, steps, warmup = 2, 1, 3
    assert bench.run_reference(Args, 2, 1) == 0       # rank 1: no work, no line
    assert capsys.readouterr().out == ""
