"""Writes tests/golden/fullsize_reaction_diffusion_b0.json: the oracle's exact
solution for instance 0 of the reaction-diffusion benchmark workload at its
full size (B = 16, 32 x 64 x 64, the workload's own data, float32-rounded as
the GPU receives them), at sampled entries.

Calls only oracle/ (and the input generator): the forward solve of Eqs. 9-10
by block elimination of A^T A with sparse LU and FP64 refinement
(oracle.solve.solve_lsq_elim, about half an hour on one core), the loss
l = mean over (b, i) of (u - target)^2 with its gradient on u,
g = 2 (u - target) / (N B), the adjoint solve of Eq. 11 with the same
factorisation and the gradients after Eq. 11 (oracle.grad).  Stored: the
relative normal-equation residual, the L2 norm of every variable block of z
and d_z, and values at seeded sample points of z, d_z, dl/dfields, dl/db.

python tests/golden/make_fullsize_golden.py
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import assemble as asm  # noqa: E402
from oracle import grad as og  # noqa: E402
from oracle import solve as osv  # noqa: E402
from paper_2502_18377_b300 import workloads as wl  # noqa: E402

OUT = os.path.join(HERE, "fullsize_reaction_diffusion_b0.json")
NSAMPLE = 1024


def main():
    t0 = time.time()
    w = wl.reaction_diffusion_2d()                 # B = 16, 32 x 64 x 64, seeds 2000 + b
    r = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)
    B, N, V = w.batch, w.npoints, 7
    b = 0
    coeff = r(w.full_coeff()[:, b])
    rhs, om, tgt = r(w.rhs[b]), r(w.omega[b]), r(w.target[b])
    A, d, kind, owner = asm.assemble(w.geom, coeff, rhs, om)
    z, lam, el = osv.solve_lsq_elim(A, d, V)
    res = osv.normal_residual(A, d, z)
    g = np.zeros(V * N)
    g[:N] = 2.0 * (z[:N] - tgt) / (N * B)
    dz, dlam = og.adjoint_elim(el, g)
    dc, db, dw = og.gradients(w.geom, A, d, kind, owner, z, lam, dz, dlam)
    # field gradients sum over the unknowns sharing a field
    F = w.fields.shape[0]
    dfields = np.stack([sum(dc[v] for v in range(V) if w.field_of[v] == f) for f in range(F)])
    rng = np.random.default_rng(20250218)
    iz = np.sort(rng.choice(V * N, NSAMPLE, replace=False))
    ip = np.sort(rng.choice(N, NSAMPLE // 2, replace=False))
    out = {
        "workload": "reaction_diffusion_2d", "batch": B, "grid": list(w.geom["n"]), "instance": b,
        "loss": "mean over (b, i) of (u - target)^2",
        "normal_residual": res,
        "adjoint_normal_residual": float(np.linalg.norm(el.At @ (el.A @ dz) - g) / np.linalg.norm(g)),
        "z_block_norms": [float(np.linalg.norm(z[v * N:(v + 1) * N])) for v in range(V)],
        "dz_block_norms": [float(np.linalg.norm(dz[v * N:(v + 1) * N])) for v in range(V)],
        "z_index": iz.tolist(), "z": z[iz].tolist(), "dz": dz[iz].tolist(),
        "point_index": ip.tolist(), "dfields": dfields[:, ip].tolist(), "drhs": db[ip].tolist(),
        "dfields_norms": [float(np.linalg.norm(x)) for x in dfields], "drhs_norm": float(np.linalg.norm(db)),
        "seconds": time.time() - t0,
    }
    with open(OUT, "w") as f:
        json.dump(out, f)
    print(f"wrote {OUT}: residual {res:.2e}, {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
