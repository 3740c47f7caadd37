"""Runs forward + MSE-gradient + adjoint steps of a benchmark workload, for
profilers (ncu) and quick timings: no clock sampling, no L2 flush, nothing
else on the GPU.

python -m paper_2502_18377_b300.profile_step [--workload transport_2d]
    [--batch B] [--grid T X Y] [--steps K] [--warmup W] [--fused-step 0|1|2|3|4]
    [--inner-iters N] [--adj-inner-iters N] [--cheb-degree M]

The environment variable MPN_TRACE makes the library print every refinement
sweep (inner iterations, update, residual, predicted error) to stderr.
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import settings
from .binding import Solver

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="transport_2d", choices=sorted(settings.BENCH_WORKLOADS))
    ap.add_argument("--batch", type=int)
    ap.add_argument("--grid", type=int, nargs=3)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--fused-step", type=int, default=3)
    ap.add_argument("--inner-iters", type=int, help="default: the workload's benchmark setting")
    ap.add_argument("--adj-inner-iters", type=int, help="default: the workload's benchmark setting")
    ap.add_argument("--cheb-degree", type=int, help="default: the workload's benchmark setting")
    a = ap.parse_args()
    w = settings.make(a.workload, batch=a.batch, grid=a.grid)
    kw = settings.solver_kwargs(a.workload)
    if a.inner_iters:
        kw["inner_iters"] = a.inner_iters
    if a.adj_inner_iters:
        kw["adj_inner_iters"] = a.adj_inner_iters
    if a.cheb_degree:
        kw["cheb_degree"] = a.cheb_degree
    dev = lambda x: torch.tensor(np.asarray(x, dtype=np.float32), device="cuda").contiguous()
    s = Solver(w.geom, w.batch, w.field_of, w.fields.shape[0], fused_step=a.fused_step, **kw)
    args = (dev(w.fields), dev(w.scalars), dev(w.rhs), dev(w.omega))
    tgt = dev(w.target)
    z = torch.empty((w.batch, s.V, w.npoints), device="cuda")

    def step():
        s.forward(*args, z=z)
        fwd = dict(s.last_stats)
        s.adjoint(*args, z, s.mse_grad(z, tgt), reuse_setup=True)
        return fwd, dict(s.last_stats)

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    s.profile(1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.steps):
        fwd, adj = step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(a.steps, 1)
    pm, pn, pb, kernels = s.profile(0)
    dom = {"us": 1e3 * pm / pn, "GBps": pb / pn / (pm / pn / 1e3) / 1e9} if pn else None
    print(json.dumps({"workload": a.workload, "batch": w.batch, "grid": list(w.geom["n"]), "ms_per_step": ms,
                      "points_per_s": w.batch * w.npoints / ms * 1e3, "levels": s.levels(), "solver_settings": kw,
                      "forward": fwd, "adjoint": adj,
                      "dominant_step": dom, "kernels_per_step": kernels / max(a.steps, 1)}))


if __name__ == "__main__":
    main()
