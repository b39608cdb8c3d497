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


def _batch_worker(rank, world, port, out):
    """One rank of the bench's sharded batch, with the oracle as the flow
    runner on tiny problems (the GPU batch's role)."""
    import sys
    import time
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from oracle import jko as ojko
    from paper_1502_06216_gb300 import inputs
    pbs = inputs.batched_problems(6, sizes=(12, 16))

    def run_share(share):
        t0 = time.perf_counter()
        flows = [ojko.problem_flow(pb, n_steps=2) for pb in share]
        secs = time.perf_counter() - t0 + 1.0 + rank      # rank 1 is the slower one
        return secs, sum(sum(f.iters) for f in flows), [f.traj[-1] for f in flows]

    idx, finals, secs_all, pairs_all = bench.sharded_batch_job(pbs, run_share)
    out.put((rank, idx, finals, secs_all, pairs_all))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharded_batch_covers_every_flow_once():
    """bench.run_batched's sharding on two gloo ranks: the shares are disjoint
    and cover the batch, every flow's result equals the same flow run alone,
    and the whole-job figures are all pairs over the slowest rank's time."""
    import sys
    import numpy as np
    sys.path.insert(0, ROOT)
    from oracle import jko as ojko
    from paper_1502_06216_gb300 import inputs
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_batch_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((out.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    pbs = inputs.batched_problems(6, sizes=(12, 16))
    alone = [ojko.problem_flow(pb, n_steps=2) for pb in pbs]
    seen = []
    for rank, idx, finals, secs_all, pairs_all in res:
        assert idx == list(range(rank, 6, 2))
        seen += idx
        for i, fin in zip(idx, finals):
            assert np.array_equal(fin, alone[i].traj[-1])
        assert pairs_all == float(sum(sum(f.iters) for f in alone))
        assert secs_all >= 2.0                               # rank 1's time is the max
    assert sorted(seen) == list(range(6))
    assert res[0][3] == res[1][3] and res[0][4] == res[1][4]  # every rank sees the same totals
