"""The benchmark's multi-GPU form is N independent replicas (no data-path
exchange): the whole-job time is the slowest rank's and the evaluations are
summed.  Checked with two gloo ranks on the CPU."""
import os
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    secs, evals = bench.combine_ranks(1.0 + rank, 10.0 * (rank + 1), world)
    out[rank] = (secs, evals)
    dist.destroy_process_group()


def test_replicas_combine_max_time_and_summed_evaluations():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank, args=(r, 2, 29517, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        assert dict(out) == {0: (2.0, 30.0), 1: (2.0, 30.0)}
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(3.5, 7.0, 1) == (3.5, 7.0)
