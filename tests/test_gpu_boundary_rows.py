"""Neumann and mixed boundary rows on the GPU (through the C ABI) against the
FP64 oracle of the same system (oracle/nonuniform.py): forward z, adjoint
d_z, the gradients (dl/domega on the Neumann / mixed faces included) and,
with per-interval steps, dl/dsteps.

Tolerances as in the other parity tests: z and d_z relative L2 <= 1e-6 per
instance, gradients relative L2 <= 1e-5.
"""
import numpy as np
import pytest
import torch

from oracle import assemble as asm
from oracle import grad as og
from oracle import nonuniform as nu
from oracle import solve as osv
from paper_2502_18377_b300 import workloads as wl

pytestmark = pytest.mark.gpu

FWD_TOL = 1e-6
GRAD_TOL = 1e-5


def _r32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _round(w, bc):
    return wl.Workload(w.name, dict(w.geom, bc=bc), list(w.field_of), _r32(w.scalars), _r32(w.fields),
                       _r32(w.rhs), _r32(w.omega), None if w.target is None else _r32(w.target))


def _dev(a):
    return torch.tensor(np.asarray(a, dtype=np.float32), device="cuda").contiguous()


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _steps(seed, w, spread):
    rng = np.random.default_rng(seed)
    return [_r32(h[None, :] * rng.uniform(1 - spread, 1 + spread, size=(w.batch, h.size)))
            for h in nu.uniform_intervals(w.geom)]


def _no_utt(w):
    w.fields[2] = 0.0
    return w


NEUMANN = (0.0, 1.0)
CASES = [
    # name, workload, boundary kinds, spread of per-interval steps (None: uniform)
    ("neumann_2d", lambda: _no_utt(wl.random_problem(51, (12, 24), (False, False), batch=2)), {1: NEUMANN}, None),
    ("mixed_2d", lambda: _no_utt(wl.random_problem(52, (10, 16), (False, False), batch=2)), {1: (0.7, -0.4)}, None),
    ("neumann_2d_final", lambda: _no_utt(wl.random_problem(53, (9, 13), (False, False), batch=2,
                                                         final_time_rows=True)), {1: NEUMANN}, None),
    ("mixed_3d", lambda: _no_utt(wl.random_problem(54, (7, 12, 10), (False, False, False), batch=2)),
     {1: NEUMANN, 2: (1.0, 0.5)}, None),
    ("neumann_y_periodic_x_3d", lambda: _no_utt(wl.random_problem(55, (6, 16, 12), (False, True, False), batch=2)),
     {2: NEUMANN}, None),
    ("c2_neumann", lambda: wl.reaction_diffusion_2d(batch=2, n=(8, 16, 16)), {1: NEUMANN, 2: NEUMANN}, None),
    ("c3_mixed", lambda: wl.linearized_burgers_1d(batch=2, n=(16, 32)), {1: (0.5, 1.0)}, None),
    ("neumann_steps_2d", lambda: _no_utt(wl.random_problem(56, (10, 20), (False, False), batch=2)),
     {1: NEUMANN}, 0.3),
    ("mixed_steps_3d", lambda: _no_utt(wl.random_problem(57, (6, 10, 12), (False, False, True), batch=2)),
     {1: (0.6, 0.8)}, 0.25),
]


def _with_open_faces(name, w):
    """The reaction-diffusion and Burgers workloads are periodic in space:
    open their axes so the boundary kinds apply."""
    if name.startswith(("c2_", "c3_")):
        w.geom = dict(w.geom, periodic=(False,) * w.ndim)
        w.omega = _r32(np.random.default_rng(9).normal(size=w.omega.shape))
    return w


@pytest.mark.parametrize("k,case", list(enumerate(CASES)), ids=[c[0] for c in CASES])
def test_boundary_rows_match_oracle(k, case):
    from paper_2502_18377_b300.binding import Solver
    name, make, bc, spread = case
    w = _round(_with_open_faces(name, make()), bc)
    V, N, F = asm.n_vars(w.ndim), w.npoints, w.fields.shape[0]
    s = Solver(w.geom, w.batch, w.field_of, F, max_refine=60, variable_steps=spread is not None)
    steps = None
    if spread is not None:
        steps = _steps(300 + k, w, spread)
        s.set_steps([_dev(h) for h in steps])
    args = (_dev(w.fields), _dev(w.scalars), _dev(w.rhs), _dev(w.omega))
    z64 = torch.empty((w.batch, V, N), device="cuda", dtype=torch.float64)
    z = s.forward(*args, z64=z64)
    g = np.random.default_rng(11).normal(size=(w.batch, V, N)).astype(np.float32)
    dz64 = torch.empty_like(z64)
    dfields, dscal, drhs, dom, dz = s.adjoint(*args, z, _dev(g), reuse_setup=True, want_dz=True, dz64=dz64)
    dsteps = [t.cpu().numpy() for t in s.step_grads(z64, dz64)] if steps is not None else None
    z, dz = z.cpu().numpy(), dz.cpu().numpy()
    dfields, dscal, drhs, dom = (t.cpu().numpy() for t in (dfields, dscal, drhs, dom))
    for b in range(w.batch):
        iv = [h[b] for h in steps] if steps is not None else None
        c = w.full_coeff()[:, b]
        A, d, kind, owner = nu.assemble(w.geom, c, w.rhs[b], w.omega[b], iv)
        zr, lam, el = osv.solve_lsq_elim(A, d, V)
        assert _rel(z[b].ravel(), zr) <= FWD_TOL, (name, b, "z", _rel(z[b].ravel(), zr))
        dzr, dlamr = og.adjoint_elim(el, g[b].astype(np.float64).ravel())
        assert _rel(dz[b].ravel(), dzr) <= FWD_TOL, (name, b, "dz", _rel(dz[b].ravel(), dzr))
        dc, db, dw = og.gradients(w.geom, A, d, kind, owner, zr, lam, dzr, dlamr)
        for f in range(F):
            ref = sum(dc[v] for v in range(V) if w.field_of[v] == f)
            assert _rel(dfields[f, b], ref) <= GRAD_TOL, (name, "field", f, _rel(dfields[f, b], ref))
        for v in range(V):
            if w.field_of[v] < 0:
                assert abs(dscal[v, b] - dc[v].sum()) <= GRAD_TOL * max(1.0, np.abs(dc[v]).sum())
        assert _rel(drhs[b], db) <= GRAD_TOL, (name, "drhs", _rel(drhs[b], db))
        assert _rel(dom[b], dw) <= GRAD_TOL, (name, "domega", _rel(dom[b], dw))
        if steps is not None:
            ivf = [h[b] for h in steps]
            dh = nu.step_gradients(w.geom, c, w.rhs[b], w.omega[b], ivf, zr, lam, dzr, dlamr)
            for ax in range(w.ndim):
                assert _rel(dsteps[ax][b], dh[ax]) <= GRAD_TOL, (name, "dsteps", ax, _rel(dsteps[ax][b], dh[ax]))


def test_reduced_operator_with_boundary_rows_matches_oracle_schur():
    from paper_2502_18377_b300.binding import Solver
    w = _round(_no_utt(wl.random_problem(58, (6, 10, 12), (False, False, False), batch=2, final_time_rows=True)),
               {1: NEUMANN, 2: (0.4, -0.7)})
    u = np.random.default_rng(0).normal(size=(w.batch, w.npoints)).astype(np.float32)
    s = Solver(w.geom, w.batch, w.field_of, w.fields.shape[0])
    q = s.apply_reduced(_dev(w.fields), _dev(w.scalars), _dev(u)).cpu().numpy()
    for b in range(w.batch):
        A, d, kind, owner = nu.assemble(w.geom, w.full_coeff()[:, b], w.rhs[b], w.omega[b])
        el = osv.solve_lsq_elim(A, d, asm.n_vars(w.ndim))[2]
        ref = el.S @ u[b].astype(np.float64)
        assert _rel(q[b], ref) <= 2e-5, _rel(q[b], ref)


def test_neumann_heat_mode_on_the_gpu():
    """u = exp(-nu k^2 t) cos(k x) with u_x = 0 at both ends, k = pi: the GPU
    solve with Neumann rows (zero data) and Dirichlet initial data converges
    to it as the grid refines (the same least-squares system as the oracle's
    stretched-grid pin, here on uniform steps)."""
    from paper_2502_18377_b300.binding import Solver
    nuv, k = 0.05, np.pi
    errs = []
    for m in (16, 32, 64):
        geom = dict(n=(m, m), step=(1.0 / (m - 1), 1.0 / (m - 1)), periodic=(False, False), stencil=3,
                    final_time_rows=False, bc={1: NEUMANN})
        t = np.arange(m) / (m - 1)
        T, X = np.meshgrid(t, t, indexing="ij")
        u = np.exp(-nuv * k * k * T) * np.cos(k * X)
        N = m * m
        fields = np.zeros((0, 1, N))
        scal = np.zeros((5, 1)); scal[1] = 1.0; scal[4] = -nuv
        om = np.zeros((1, N)); om[0, :m] = u[0]          # t = 0 face; Neumann faces take 0
        s = Solver(geom, 1, [-1] * 5, 0, max_refine=60)
        z = s.forward(None, _dev(scal), _dev(np.zeros((1, N))), _dev(om)).cpu().numpy()
        errs.append(np.linalg.norm(z[0, 0] - u.ravel()) / np.linalg.norm(u))
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[2] < 2e-3, errs
