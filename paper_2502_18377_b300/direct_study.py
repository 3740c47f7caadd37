"""Direct path against multigrid-preconditioned CG on small problems.

    python -m paper_2502_18377_b300.direct_study

For the advection-diffusion workload (B = 4, 32 x 32, scalar coefficients,
Dirichlet x) and Laplace's equation (B = 32, 32 x 32): wall time of one
forward solve and of one forward + adjoint step (CUDA events, after warm-up)
through the direct path (whole reduced system factorised, explicit inverse
applied once per refinement sweep) and through the multigrid path, with the
refinement sweeps, and the largest relative difference between the two FP32
solutions.  Prints one JSON line per workload.
"""
import json

import numpy as np
import torch

from . import workloads as wl
from .binding import Solver


def _time(fn, reps=5):
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def compare(w, **kw):
    dev = lambda a: torch.tensor(np.asarray(a, dtype=np.float32), device="cuda")
    F = w.fields.shape[0]
    args = (dev(w.fields) if F else torch.zeros((1,), device="cuda"), dev(w.scalars), dev(w.rhs), dev(w.omega))
    g = torch.randn((w.batch, 2 * w.ndim + 1, w.npoints), device="cuda", generator=torch.Generator("cuda").manual_seed(0))
    out = {"workload": w.name, "batch": w.batch, "grid": list(w.geom["n"])}
    zs = {}
    for name, direct in (("direct", True), ("multigrid", False)):
        s = Solver(w.geom, w.batch, w.field_of, F, direct=direct, **({} if direct else kw))
        z = torch.empty((w.batch, 2 * w.ndim + 1, w.npoints), device="cuda")
        fwd = lambda: s.forward(*args, z=z)
        def step():
            s.forward(*args, z=z)
            s.adjoint(*args, z, g, reuse_setup=True)
        t_f = _time(fwd)
        sweeps = s.last_stats["sweeps"]
        t_s = _time(step)
        zs[name] = z.clone()
        out[name] = {"forward_ms": t_f, "forward_adjoint_ms": t_s, "sweeps": sweeps, "levels": len(s.levels())}
    d = (zs["direct"] - zs["multigrid"]).flatten(1).norm(dim=1) / zs["multigrid"].flatten(1).norm(dim=1)
    out["max_rel_diff"] = float(d.max())
    return out


def main():
    print(json.dumps(compare(wl.advection_diffusion_1d())), flush=True)
    print(json.dumps(compare(wl.laplace_2d(batch=32, n=32), coarsen_time=True)), flush=True)


if __name__ == "__main__":
    main()
