"""Runs forward + MSE-gradient + adjoint steps of a benchmark workload, for
profilers (ncu) and quick timings: no clock sampling, no L2 flush, nothing
else on the GPU.

python -m paper_2502_18377_b300.profile_step [--workload transport_2d]
    [--batch B] [--grid T X Y] [--steps K] [--warmup W] [--fused-step 0|1|2]
    [--inner-iters N] [--cheb-degree M]

The environment variable MPN_TRACE makes the library print every refinement
sweep (inner iterations, update, residual, predicted error) to stderr.
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import workloads as wl
from .binding import Solver

WORKLOADS = {
    "transport_2d": (wl.transport_2d, 4, (32, 256, 256)),
    "reaction_diffusion_2d_64x128x128": (wl.reaction_diffusion_2d, 8, (64, 128, 128)),
    "reaction_diffusion_2d": (wl.reaction_diffusion_2d, 16, (32, 64, 64)),
}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="transport_2d", choices=sorted(WORKLOADS))
    ap.add_argument("--batch", type=int)
    ap.add_argument("--grid", type=int, nargs=3)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--fused-step", type=int, default=1)
    ap.add_argument("--inner-iters", type=int, default=5)
    ap.add_argument("--cheb-degree", type=int, default=5)
    a = ap.parse_args()
    gen, b0, g0 = WORKLOADS[a.workload]
    w = gen(batch=a.batch or b0, n=tuple(a.grid) if a.grid else g0)
    dev = lambda x: torch.tensor(np.asarray(x, dtype=np.float32), device="cuda").contiguous()
    s = Solver(w.geom, w.batch, w.field_of, w.fields.shape[0], fused_step=a.fused_step,
               inner_iters=a.inner_iters, cheb_degree=a.cheb_degree)
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
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.steps):
        fwd, adj = step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(a.steps, 1)
    print(json.dumps({"workload": a.workload, "batch": w.batch, "grid": list(w.geom["n"]), "ms_per_step": ms,
                      "points_per_s": w.batch * w.npoints / ms * 1e3, "levels": s.levels(),
                      "forward": fwd, "adjoint": adj}))


if __name__ == "__main__":
    main()
