"""The benchmark workloads and the solver settings measured best for each.

One table serves the benchmark, the profiling driver and the full-size
tests, so all three run the same launch configuration.  The settings are
solver parameters only (smoother degree and inner iterations per refinement
sweep, forward and adjoint); they change the speed, never the solution, which every setting
drives to the same tolerance.  They were chosen by timing forward + adjoint
steps on one B300 (figures in the design notes):

* transport (advection-dominated, cell Peclet number ~25): point smoothing
  reduces the error slowly per V-cycle, so longer inner solves with a
  cheaper V-cycle win: Chebyshev degree 3, 25 CG iterations per sweep
  (215 ms per step against 316 ms with degree 5 and 5 iterations).  The
  forward solve takes 27 iterations per sweep and the adjoint 30: three
  sweeps each on every seeded batch tried (25 left one of four batches at
  four forward sweeps, 169.9 ms; the adjoint's rougher right-hand side
  needed four sweeps at 25 and 28 iterations, 155.1 and 162.5 ms, three at
  30, 144.5 ms with 25 forward iterations);
* reaction-diffusion at 64 x 128 x 128: degree 4, 8 iterations (79 ms
  against 92 ms);
* linearized Burgers at 128 x 256 (time is never coarsened and its coupling
  along t is strong, so the V-cycle is weak there and CG needs long inner
  solves): degree 5, 30 iterations, three sweeps each way (152.7 ms per
  step against 210.2 ms with 5 iterations, where short sweeps gaining less
  than a digit grow to 7 sweeps; 20 iterations 174.4 ms, 40 198.7 ms);
* reaction-diffusion at 32 x 64 x 64 and advection-diffusion at 32 x 32:
  the library defaults (degree 5, 5 iterations).
"""
from __future__ import annotations

from . import workloads as wl

# name -> (generator, batch per GPU, grid, seed base, solver keyword arguments)
BENCH_WORKLOADS = {
    "transport_2d": (wl.transport_2d, 4, (32, 256, 256), 5000, dict(cheb_degree=3, inner_iters=27,
                                                                    adj_inner_iters=30)),
    "reaction_diffusion_2d_64x128x128": (wl.reaction_diffusion_2d, 8, (64, 128, 128), 4000,
                                         dict(cheb_degree=4, inner_iters=8)),
    "reaction_diffusion_2d": (wl.reaction_diffusion_2d, 16, (32, 64, 64), 2000, dict()),
    # the two 1-D+t families (L2-resident: absolute throughput only)
    "linearized_burgers_1d": (wl.linearized_burgers_1d, 32, (128, 256), 3000, dict(inner_iters=30)),
    "advection_diffusion_1d": (wl.advection_diffusion_1d, 4, (32, 32), 1000, dict()),
}


def make(name, batch=None, grid=None, seed_offset=0):
    """The workload `name` (optionally at another batch or grid)."""
    gen, b0, g0, seed, _ = BENCH_WORKLOADS[name]
    return gen(batch=batch or b0, n=tuple(grid) if grid else g0, seed_base=seed + seed_offset)


def solver_kwargs(name):
    return dict(BENCH_WORKLOADS[name][4])
