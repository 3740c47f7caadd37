"""Multi-rank host logic of bench.py on two CPU ranks (gloo, 127.0.0.1).

The batch shards across ranks with no data-path collective: every rank
generates and solves a batch of its own (distinct seeds), the step time of the
job is the maximum over ranks, and the reported throughput counts the points
of all ranks.  A rank that raises is seen by the parent as a failed process.
"""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q, fail_rank):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        if rank == fail_rank:
            raise RuntimeError("rank failure injected on the host")
        import bench
        w, fields, scal, rhs, om, tgt = bench.make_inputs(rank, batch=2, grid=(4, 8, 8))
        ms = bench.job_time_ms(10.0 + 3.0 * rank, world)
        value = bench.job_throughput(world, 2, w.npoints, ms)
        q.put((rank, float(np.abs(tgt).sum()), float(np.abs(fields).sum()), ms, value, w.npoints))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _run(world, fail_rank=-1):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q, fail_rank)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    for p in procs:                 # a rank still waiting after the timeout: end it (our own child)
        if p.is_alive():
            p.terminate()
            p.join(timeout=10)
    codes = [p.exitcode for p in procs]
    out = []
    while not q.empty():
        out.append(q.get())
    return codes, sorted(out)


def test_two_ranks_shard_batches_and_take_the_slowest_rank():
    codes, out = _run(2)
    assert codes == [0, 0], codes
    assert len(out) == 2
    (r0, tgt0, f0, ms0, v0, n), (r1, tgt1, f1, ms1, v1, _) = out
    # each rank has its own batch
    assert tgt0 != tgt1 and f0 != f1
    # the job's step time is the slowest rank's, on every rank
    assert ms0 == ms1 == 13.0
    # throughput counts both ranks' points
    assert abs(v0 - 2 * 2 * n / 13e-3) < 1e-6 * v0 and v0 == v1


def test_a_failing_rank_is_reported_not_hung():
    """A rank that raises before the collective: it exits non-zero and the
    other rank ends (its collective errors out or completes) within the join
    timeout instead of hanging the job."""
    codes, out = _run(2, fail_rank=1)
    assert codes[1] != 0
    assert all(c is not None for c in codes), codes
