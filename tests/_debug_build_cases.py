"""Solver runs shared by the bounds-checked build's test (not collected by
pytest): forward z, the MSE-loss adjoint (d_z and dl/db) and the reduced
operator apply on small problems whose kernels cover the checked index
helpers: 1-D + t float4 levels (Dirichlet and periodic x, final-time rows),
scalar two-pass levels, 3-D float4 two-pass levels, the fused tile step,
Neumann rows and per-interval steps.

Run as a script (`python _debug_build_cases.py LIB OUT.npz`) it loads the
library at LIB before anything else and saves every result and the
library's recorded index-check code per case to OUT.npz.
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _no_utt(w):
    w.fields[2] = 0.0
    return w


def cases():
    from paper_2502_18377_b300 import workloads as wl
    return [
        # name, workload, solver keyword arguments, boundary kinds, per-interval step spread
        ("adv_1d", lambda: wl.advection_diffusion_1d(), {}, None, None),
        ("burgers_1d", lambda: wl.linearized_burgers_1d(batch=2, n=(32, 64)), {}, None, None),
        ("final_2d", lambda: _no_utt(wl.random_problem(28, (9, 16), (False, False), batch=2,
                                                       final_time_rows=True)), {}, None, None),
        ("odd_2d", lambda: wl.random_problem(22, (9, 13), (False, False), batch=2, final_time_rows=True),
         {}, None, None),
        ("rd_fused", lambda: wl.reaction_diffusion_2d(batch=2, n=(8, 16, 16)), {}, None, None),
        ("rd_twopass", lambda: wl.reaction_diffusion_2d(batch=2, n=(8, 16, 16)), {"fused_step": 0}, None, None),
        ("transport", lambda: wl.transport_2d(batch=2, n=(8, 16, 16)), {}, None, None),
        ("mixed_3d", lambda: _no_utt(wl.random_problem(23, (7, 16, 12), (False, True, False), batch=2)),
         {}, None, None),
        ("neumann_2d", lambda: _no_utt(wl.random_problem(51, (12, 24), (False, False), batch=2)), {},
         {1: (0.0, 1.0)}, None),
        ("steps_2d", lambda: _no_utt(wl.random_problem(54, (10, 16), (False, True), batch=2)),
         {"variable_steps": True}, None, 0.3),
    ]


def run():
    """Every case's results (float64 arrays) and index-check codes."""
    import torch
    from oracle import nonuniform as nu
    from paper_2502_18377_b300.binding import Solver
    dev = lambda a: torch.tensor(np.asarray(a, dtype=np.float32), device="cuda").contiguous()
    out = {}
    for name, make, kw, bc, spread in cases():
        w = make()
        geom = dict(w.geom, bc=bc) if bc else w.geom
        s = Solver(geom, w.batch, w.field_of, w.fields.shape[0], max_refine=60, **kw)
        if spread is not None:
            rng = np.random.default_rng(7)
            s.set_steps([dev(h[None, :] * rng.uniform(1 - spread, 1 + spread, size=(w.batch, h.size)))
                         for h in nu.uniform_intervals(w.geom)])
        args = (dev(w.fields), dev(w.scalars), dev(w.rhs), dev(w.omega))
        tgt = dev(w.target if w.target is not None
                  else w.omega + 0.1 * np.random.default_rng(3).standard_normal(w.omega.shape))
        z = s.forward(*args)
        gz = s.mse_grad(z, tgt)
        _, _, drhs, _, dz = s.adjoint(*args, z, gz, reuse_setup=True, want_dz=True)
        u = dev(np.random.default_rng(5).standard_normal((w.batch, w.npoints)))
        q = s.apply_reduced(args[0], args[1], u)
        torch.cuda.synchronize()
        code = s.debug_take()
        out[name + ":z"] = z.double().cpu().numpy()
        out[name + ":dz"] = dz.double().cpu().numpy()
        out[name + ":drhs"] = drhs.double().cpu().numpy()
        out[name + ":q"] = q.double().cpu().numpy()
        out[name + ":code"] = np.array(-1 if code is None else code)
        del s
    return out


if __name__ == "__main__":
    from paper_2502_18377_b300 import binding
    binding.load(sys.argv[1])
    np.savez(sys.argv[2], **run())
