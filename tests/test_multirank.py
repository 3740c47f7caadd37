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


def _grad_worker(rank, world, port, q, leave_after):
    """Linear least squares on a shard of a fixed batch: the all-reduced mean
    of the per-rank gradients must equal the full-batch gradient.  With
    leave_after >= 0, rank 1 leaves after that many steps and rank 0 must
    see its next collective fail, not hang."""
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import datetime
    import torch
    import torch.distributed as dist
    from paper_2502_18377_b300.warmstart import allreduce_mean
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    g = torch.Generator().manual_seed(3)
    X = torch.randn(8, 3, generator=g, dtype=torch.float64)
    y = torch.randn(8, generator=g, dtype=torch.float64)
    w = torch.randn(3, generator=g, dtype=torch.float64)
    b = torch.zeros(1, dtype=torch.float64)
    shard = slice(4 * rank, 4 * rank + 4)
    try:
        for step in range(3):
            if leave_after >= 0 and rank == 1 and step == leave_after:
                return                                  # leaves between steps
            Xr, yr = X[shard], y[shard]
            res = Xr @ w + b - yr
            gw = 2.0 / Xr.shape[0] * Xr.T @ res          # gradient of this rank's mean loss
            gb = (2.0 / Xr.shape[0] * res.sum()).reshape(1)
            allreduce_mean([gw, gb])
            full = X @ w + b - y
            ok = bool(torch.allclose(gw, 2.0 / 8 * X.T @ full, rtol=1e-12, atol=1e-12) and
                      torch.allclose(gb, (2.0 / 8 * full.sum()).reshape(1), rtol=1e-12, atol=1e-12))
            q.put((rank, step, ok, ""))
            w = w - 0.1 * gw
            b = b - 0.1 * gb
    except Exception as e:                              # the collective failed: report it
        q.put((rank, -1, False, type(e).__name__))
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def _run_grad(world, leave_after):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_grad_worker, args=(r, world, port, q, leave_after)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    for p in procs:
        if p.is_alive():
            p.terminate()
            p.join(timeout=10)
    out = []
    while not q.empty():
        out.append(q.get())
    return [p.exitcode for p in procs], sorted(out)


def test_gradient_allreduce_equals_full_batch_gradient():
    codes, out = _run_grad(2, -1)
    assert codes == [0, 0], codes
    assert len(out) == 6 and all(ok for _, _, ok, _ in out), out


def test_rank_leaving_between_steps_is_reported():
    codes, out = _run_grad(2, 1)
    assert codes == [0, 0], codes
    steps0 = [s for r, s, ok, _ in out if r == 0]
    assert 0 in steps0                                  # the first step ran on both ranks
    assert any(r == 0 and s == -1 and err for r, s, ok, err in out), out   # rank 0 saw the failure
