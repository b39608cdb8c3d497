"""The N > 1 host path of bench.py on the CPU: two ranks over gloo.

With N GPUs the benchmark runs N independent replicas of the workload (one
flow per rank, no data exchange between ranks): the whole-job rate is the
pairs all ranks ran over the slowest rank's time.  These tests run that
aggregation, and the rank rules of the reference arm, as two processes."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r, local = bench.dist_env()
    total_s, iters = bench.aggregate_over_ranks(1.0 + 0.5 * rank, 100 * (rank + 1), ws)
    # the reference arm: rank 0 alone runs and prints; the others return 0
    ref_rc = bench.run_reference(type("A", (), {"n": 16, "steps": 1, "warmup": 0})()) \
        if rank != 0 else None
    out.put((rank, ws, r, local, total_s, iters, ref_rc))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_and_reference_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ws, r, local, total_s, iters, ref_rc in res:
        assert (ws, r, local) == (2, rank, rank)
        assert total_s == 1.5          # the slowest rank's seconds
        assert iters == 300.0          # pairs of both ranks
        if rank == 1:
            assert ref_rc == 0         # no work on ranks > 0


def test_one_rank_is_the_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_over_ranks(2.5, 7, 1) == (2.5, 7.0)
