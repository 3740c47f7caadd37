"""Laplace solver study: the paper's solver unit test and its time / memory
table (2-D Laplace equation, batch 32, multigrid-preconditioned solve at 32^2,
64^2 and 128^2), run through the library on one GPU.

    python -m paper_2502_18377_b300.laplace_study [--batch 32] [--sizes 32 64 128] [--keep-time-axis]

The hierarchy halves both axes (coarsen_time), since Laplace's equation is
elliptic in the first axis too.

Prints one JSON line per grid and inner solver: wall time of one forward solve
(CUDA events, after warm-up), device memory of the problem (the library's
workspace plus the caller's input and output tensors), refinement sweeps and
inner iterations, and the relative L2 error of u against the harmonic function
the boundary data come from (discretisation error; the solve itself meets the
1e-7 refinement tolerance).  The paper's figures (its own hardware): 1.6 GB /
6.16 s, 4.63 GB / 13.9 s, 16.7 GB / 33.9 s.
"""
import argparse
import json

import numpy as np
import torch

from . import workloads as wl
from .binding import Solver


def run(n, batch, krylov, coarsen_time, reps=3):
    w = wl.laplace_2d(batch=batch, n=n)
    dev = lambda a: torch.tensor(np.asarray(a, dtype=np.float32), device="cuda")
    args = (torch.zeros((1,), device="cuda"), dev(w.scalars), dev(w.rhs), dev(w.omega))
    s = Solver(w.geom, batch, w.field_of, 0, krylov=krylov, max_refine=60, coarsen_time=coarsen_time)
    z = torch.empty((batch, 5, w.npoints), device="cuda")
    s.forward(*args, z=z)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        s.forward(*args, z=z)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    u = z[:, 0].double().cpu().numpy()
    ref = w.target
    err = float(np.max(np.linalg.norm(u - ref, axis=1) / np.linalg.norm(ref, axis=1)))
    io_bytes = sum(t.numel() * t.element_size() for t in args) + z.numel() * 4
    return {"grid": [n, n], "batch": batch, "krylov": krylov, "coarsen_time": coarsen_time, "time_s": ms / 1e3,
            "memory_gb": (s.workspace_bytes + io_bytes) / 1e9, "levels": s.levels(),
            "sweeps": s.last_stats["sweeps"], "inner_iters": s.last_stats["pcg_iters"],
            "rel_l2_vs_harmonic": err}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--sizes", type=int, nargs="+", default=[32, 64, 128])
    ap.add_argument("--krylov", nargs="+", default=["cg", "fgmres"])
    ap.add_argument("--keep-time-axis", action="store_true",
                    help="do not halve the first axis in the hierarchy (the setting for time-dependent problems)")
    a = ap.parse_args()
    for n in a.sizes:
        for kr in a.krylov:
            print(json.dumps(run(n, a.batch, kr, not a.keep_time_axis)), flush=True)


if __name__ == "__main__":
    main()
