"""Learned warm start at the scale of its workload: train the 3x3x3
convolutional network on solves of the plain method, then compare held-out
solves with and without its prediction.

Workload: reaction-diffusion 2D+t, batch 8, grid 64 x 128 x 128, periodic in
x and y (the benchmark's second workload and its solver settings).
Training: `--train` seeded instances (seeds 100000 + k) solved by the plain
multigrid-preconditioned solve to its tolerance, the network fitted to u by
Adam for `--epochs` epochs in a seeded order.  Held out: `--heldout`
instances (seeds 200000 + k, disjoint).  For each held-out batch: the cold
solve (u0 = 0) and the warm solve (u0 = the network's prediction) to the
same tolerance, their refinement sweeps, CG iterations and times (CUDA
events; the warm time includes the network's inference), the prediction's
relative error, and the agreement of the two solutions.

Inputs are drawn on the host by the shared generator, in a process pool
started (spawn) before any CUDA call, while the GPU solves earlier batches.

Plain FP32 multigrid-CG (one sweep of k FP32 CG iterations, no FP64
refinement) is timed on the first held-out batches against the mixed solve,
with its error against the mixed solve's solution.

python -m paper_2502_18377_b300.warmstart_study [--train 2000] [--heldout 200]
    [--epochs 8] [--plain-iters 10,20,40,80] [--workers 16] [--out FILE.json]
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import time

import numpy as np

BATCH = 8
GRID = (64, 128, 128)
TRAIN_SEED, HELDOUT_SEED = 100_000, 200_000


def _inputs(seed_base):
    """One batch of the workload (float32 arrays), drawn on the host."""
    from paper_2502_18377_b300 import workloads as wl
    w = wl.reaction_diffusion_2d(batch=BATCH, n=GRID, seed_base=seed_base)
    f32 = lambda a: np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    return seed_base, f32(w.fields), f32(w.scalars), f32(w.rhs), f32(w.omega)


def _batches(pool, first_seed, count):
    """Batches of `count` instances (rounded up to whole batches) in order."""
    seeds = [first_seed + BATCH * k for k in range((count + BATCH - 1) // BATCH)]
    return pool.imap(_inputs, seeds)


def _solve_timed(torch, s, args, u0=None):
    """One forward solve timed with CUDA events; returns (z, ms, stats)."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    z = s.forward(*args, u0=u0)
    e1.record()
    torch.cuda.synchronize()
    return z, e0.elapsed_time(e1), dict(s.last_stats)


def run(a, pool):
    import torch

    from . import settings
    from .binding import Solver
    from .warmstart import WarmStartNet, WarmStartTrainer

    torch.cuda.set_device(0)
    dev = lambda x: torch.from_numpy(x).cuda()
    geom = None
    s = None
    # 1. training data: plain-method solves of the training instances
    train, gen_wait = [], 0.0
    t0 = time.time()
    it = _batches(pool, TRAIN_SEED, a.train)
    while True:
        tw = time.time()
        try:
            seed, fields, scal, rhs, om = next(it)
        except StopIteration:
            break
        gen_wait += time.time() - tw
        if s is None:
            from . import workloads as wl
            w0 = wl.reaction_diffusion_2d(batch=1, n=GRID, seed_base=seed)
            geom, field_of = w0.geom, w0.field_of
            s = Solver(geom, BATCH, field_of, fields.shape[0],
                       **settings.solver_kwargs("reaction_diffusion_2d_64x128x128"))
        args = (dev(fields), dev(scal), dev(rhs), dev(om))
        z = s.forward(*args)
        train.append((args[0], args[2], z[:, 0].contiguous()))
    torch.cuda.synchronize()
    t_data = time.time() - t0
    print(f"training data: {len(train)} batches of {BATCH} in {t_data:.1f} s "
          f"({gen_wait:.1f} s waiting for the host generator)", flush=True)

    # 2. training
    net = WarmStartNet(geom, BATCH, 2, seed=a.seed, lr=a.lr)
    net.fit_scales(*train[0])
    trainer = WarmStartTrainer(net, train, seed=a.seed)
    curve = []
    t0 = time.time()
    for ep in range(a.epochs):
        tot = torch.zeros((), device="cuda")
        for _ in range(len(train)):
            tot += trainer.step()
        curve.append(float(tot) / len(train))
        print(f"epoch {ep}: mean loss {curve[-1]:.4e} ({time.time() - t0:.1f} s)", flush=True)
    torch.cuda.synchronize()
    t_train = time.time() - t0
    steps = a.epochs * len(train)
    return s, net, train, dict(train_instances=len(train) * BATCH, epochs=a.epochs, steps=steps,
                               data_seconds=t_data, train_seconds=t_train,
                               ms_per_train_step=1e3 * t_train / max(steps, 1), loss_curve=curve)


def evaluate(a, pool, s, net):
    """Cold and warm solves of the held-out batches."""
    import torch
    dev = lambda x: torch.from_numpy(x).cuda()
    rows = []
    warm_up = True
    for seed, fields, scal, rhs, om in _batches(pool, HELDOUT_SEED, a.heldout):
        args = (dev(fields), dev(scal), dev(rhs), dev(om))
        if warm_up:                      # capture the sweep graphs of both paths once, untimed
            z = s.forward(*args)
            s.forward(*args, u0=net.predict(args[0], args[2]).clone())
            warm_up = False
        z_cold, ms_cold, st_cold = _solve_timed(torch, s, args)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        u0 = net.predict(args[0], args[2])
        e1.record()
        z_warm, ms_solve, st_warm = _solve_timed(torch, s, args, u0=u0)
        ms_pred = e0.elapsed_time(e1)
        u = z_cold[:, 0]
        rows.append(dict(seed=seed, ms_cold=ms_cold, ms_warm=ms_pred + ms_solve, ms_predict=ms_pred,
                         sweeps_cold=st_cold["sweeps"], sweeps_warm=st_warm["sweeps"],
                         iters_cold=st_cold["pcg_iters"], iters_warm=st_warm["pcg_iters"],
                         pred_error=float((u0 - u).norm() / u.norm()),
                         agreement=float((z_warm - z_cold).norm() / z_cold.norm())))
    tot = lambda k: float(sum(r[k] for r in rows))
    return dict(heldout_instances=len(rows) * BATCH, batches=len(rows),
                ms_cold=tot("ms_cold"), ms_warm=tot("ms_warm"), ms_predict=tot("ms_predict"),
                speedup=tot("ms_cold") / tot("ms_warm"),
                iters_cold=tot("iters_cold"), iters_warm=tot("iters_warm"),
                sweeps_cold=tot("sweeps_cold"), sweeps_warm=tot("sweeps_warm"),
                pred_error_mean=float(np.mean([r["pred_error"] for r in rows])),
                agreement_max=float(max(r["agreement"] for r in rows)), per_batch=rows)


def plain_fp32(a, pool, net_solver_kwargs):
    """Plain FP32 multigrid-preconditioned CG (no FP64 refinement: one sweep
    of k CG iterations from zero, max_refine = 1) on the first held-out
    batches, against the refined mixed-precision solve of the same data:
    relative L2 error of the whole z and of u (max over instances), time."""
    import torch

    from .binding import Solver
    dev = lambda x: torch.from_numpy(x).cuda()
    ks = [int(k) for k in a.plain_iters.split(",")]
    out = {k: dict(iters=k, ms=0.0, err_z=0.0, err_u=0.0) for k in ks}
    ref = dict(ms=0.0)
    s_ref = None
    for nb, (seed, fields, scal, rhs, om) in enumerate(_batches(pool, HELDOUT_SEED, BATCH * a.plain_batches)):
        args = (dev(fields), dev(scal), dev(rhs), dev(om))
        from . import workloads as wl
        if s_ref is None:
            w0 = wl.reaction_diffusion_2d(batch=1, n=GRID, seed_base=seed)
            s_ref = Solver(w0.geom, BATCH, w0.field_of, 2, **net_solver_kwargs)
            plain = {k: Solver(w0.geom, BATCH, w0.field_of, 2, max_refine=1,
                               **dict(net_solver_kwargs, inner_iters=k)) for k in ks}
            s_ref.forward(*args)
            for k in ks:
                plain[k].forward(*args, allow_not_converged=True)
        z_ref, ms, _ = _solve_timed(torch, s_ref, args)
        ref["ms"] += ms
        for k in ks:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            z = plain[k].forward(*args, allow_not_converged=True)
            e1.record()
            torch.cuda.synchronize()
            o = out[k]
            o["ms"] += e0.elapsed_time(e1)
            dzb = (z - z_ref).reshape(BATCH, -1).norm(dim=1) / z_ref.reshape(BATCH, -1).norm(dim=1)
            dub = (z[:, 0] - z_ref[:, 0]).norm(dim=1) / z_ref[:, 0].norm(dim=1)
            o["err_z"] = max(o["err_z"], float(dzb.max()))
            o["err_u"] = max(o["err_u"], float(dub.max()))
    return dict(batches=a.plain_batches, mixed_ms=ref["ms"], plain=[out[k] for k in ks])


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--heldout", type=int, default=200)
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--workers", type=int, default=min(16, os.cpu_count() or 1))
    ap.add_argument("--plain-iters", default="10,20,40,80")
    ap.add_argument("--plain-batches", type=int, default=4)
    ap.add_argument("--out")
    a = ap.parse_args()
    # the pool starts (spawn) before any CUDA call in this process
    with mp.get_context("spawn").Pool(a.workers) as pool:
        s, net, train, tr = run(a, pool)
        del train
        ev = evaluate(a, pool, s, net)
        from . import settings
        pl = plain_fp32(a, pool, settings.solver_kwargs("reaction_diffusion_2d_64x128x128"))
    out = dict(workload="reaction_diffusion_2d", batch=BATCH, grid=list(GRID), training=tr, heldout=ev,
               plain_fp32_mgcg=pl)
    line = json.dumps(out)
    print(line, flush=True)
    if a.out:
        with open(a.out, "w") as f:
            f.write(line + "\n")


if __name__ == "__main__":
    main()
