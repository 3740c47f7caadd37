"""Per-interval steps on the GPU (through the C ABI) against the FP64 oracle
of the same system (oracle/nonuniform.py): forward z, adjoint d_z, the
coefficient / right-hand-side / boundary gradients and dl/dsteps.

Both sides receive the same float32-rounded seeded inputs and steps.
Tolerances as in the uniform parity tests: z and d_z relative L2 <= 1e-6 per
instance; gradients relative L2 <= 1e-5 (dl/dsteps per axis).
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


def _round(w):
    return wl.Workload(w.name, w.geom, list(w.field_of), _r32(w.scalars), _r32(w.fields), _r32(w.rhs),
                       _r32(w.omega), None if w.target is None else _r32(w.target))


def _dev(a, dtype=np.float32):
    return torch.tensor(np.asarray(a, dtype=dtype), device="cuda").contiguous()


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _steps(seed, w, spread):
    """Per-instance intervals around the uniform step, float32-rounded:
    one array [B, m_d] per axis."""
    rng = np.random.default_rng(seed)
    out = []
    for h in nu.uniform_intervals(w.geom):
        out.append(_r32(h[None, :] * rng.uniform(1 - spread, 1 + spread, size=(w.batch, h.size))))
    return out


def _stretched_steps(w):
    """A smooth stretching x = s + 0.08 sin(2 pi s) of every open axis (the
    same for every instance), uniform periodic axes scaled per instance."""
    out = []
    for d, h in enumerate(nu.uniform_intervals(w.geom)):
        if w.geom["periodic"][d]:
            sc = 1.0 + 0.1 * np.arange(w.batch)[:, None]
            out.append(_r32(np.broadcast_to(h[None, :], (w.batch, h.size)) * sc))
        else:
            L = h.sum()
            s = np.linspace(0.0, 1.0, h.size + 1)
            x = L * (s + 0.08 * np.sin(2 * np.pi * s))
            out.append(_r32(np.broadcast_to(np.diff(x)[None, :], (w.batch, h.size))))
    return out


def _solver(w, **kw):
    from paper_2502_18377_b300.binding import Solver
    kw.setdefault("max_refine", 60)
    return Solver(w.geom, w.batch, w.field_of, w.fields.shape[0], variable_steps=True, **kw)


def _oracle(w, steps, b):
    iv = [h[b] for h in steps]
    c = w.full_coeff()[:, b]
    A, d, kind, owner = nu.assemble(w.geom, c, w.rhs[b], w.omega[b], iv)
    z, lam, el = osv.solve_lsq_elim(A, d, asm.n_vars(w.ndim))
    return A, d, kind, owner, z, lam, el, iv, c


def _no_utt(w):
    w.fields[2] = 0.0
    return w


CASES = [
    ("rand_dirichlet_2d", lambda: _no_utt(wl.random_problem(41, (12, 24), (False, False), batch=2)), 0.3),
    ("rand_periodic_2d", lambda: _no_utt(wl.random_problem(42, (10, 16), (False, True), batch=2)), 0.3),
    ("rand_final_2d", lambda: _no_utt(wl.random_problem(43, (9, 13), (False, False), batch=2,
                                                      final_time_rows=True)), 0.25),
    ("rand_mixed_3d", lambda: _no_utt(wl.random_problem(44, (7, 16, 12), (False, True, False), batch=2)), 0.3),
    ("c2_small", lambda: wl.reaction_diffusion_2d(batch=2, n=(8, 16, 16)), 0.3),
    ("c5_small", lambda: wl.transport_2d(batch=2, n=(8, 16, 16)), 0.2),
    ("c3_small", lambda: wl.linearized_burgers_1d(batch=2, n=(16, 32)), 0.3),
    ("laplace_24", lambda: wl.laplace_2d(batch=2, n=24), 0.3),
]


def _steps_for(name, w, spread, k):
    return _steps(100 + k, w, spread)


@pytest.mark.parametrize("k,case", list(enumerate(CASES)), ids=[c[0] for c in CASES])
def test_forward_adjoint_and_gradients_match_oracle(k, case):
    name, make, spread = case
    w = _round(make())
    steps = _steps_for(name, w, spread, k)
    kw = dict(coarsen_time=True) if name.startswith("laplace") else {}
    s = _solver(w, **kw)
    s.set_steps([_dev(h) for h in steps])
    args = (_dev(w.fields), _dev(w.scalars), _dev(w.rhs), _dev(w.omega))
    V, N, F = asm.n_vars(w.ndim), w.npoints, w.fields.shape[0]
    z64 = torch.empty((w.batch, V, N), device="cuda", dtype=torch.float64)
    z = s.forward(*args, z64=z64)
    rng = np.random.default_rng(7)
    g = rng.normal(size=(w.batch, V, N)).astype(np.float32)
    dz64 = torch.empty_like(z64)
    dfields, dscal, drhs, dom, dz = s.adjoint(*args, z, _dev(g), reuse_setup=True, want_dz=True, dz64=dz64)
    dsteps = [t.cpu().numpy() for t in s.step_grads(z64, dz64)]
    z, dz = z.cpu().numpy(), dz.cpu().numpy()
    dfields, dscal, drhs, dom = (t.cpu().numpy() for t in (dfields, dscal, drhs, dom))
    for b in range(w.batch):
        A, d, kind, owner, zr, lam, el, iv, c = _oracle(w, steps, b)
        assert _rel(z[b].ravel(), zr) <= FWD_TOL, (name, b, "z", _rel(z[b].ravel(), zr))
        assert _rel(z[b, 0], zr[:N]) <= FWD_TOL, (name, b, "u")
        dzr, dlamr = og.adjoint_elim(el, g[b].astype(np.float64).ravel())
        assert _rel(dz[b].ravel(), dzr) <= FWD_TOL, (name, b, "dz", _rel(dz[b].ravel(), dzr))
        dc, db, dw = og.gradients(w.geom, A, d, kind, owner, zr, lam, dzr, dlamr)
        for f in range(F):
            ref = sum(dc[v] for v in range(V) if w.field_of[v] == f)
            assert _rel(dfields[f, b], ref) <= GRAD_TOL, (name, "field", f, _rel(dfields[f, b], ref))
        for v in range(V):
            if w.field_of[v] < 0:
                assert abs(dscal[v, b] - dc[v].sum()) <= GRAD_TOL * max(1.0, np.abs(dc[v]).sum())
        assert _rel(drhs[b], db) <= GRAD_TOL
        assert _rel(dom[b], dw) <= GRAD_TOL
        dh = nu.step_gradients(w.geom, c, w.rhs[b], w.omega[b], iv, zr, lam, dzr, dlamr)
        for ax in range(w.ndim):
            assert _rel(dsteps[ax][b], dh[ax]) <= GRAD_TOL, (name, b, "dsteps", ax, _rel(dsteps[ax][b], dh[ax]))


def test_stretched_grid_forward_matches_oracle():
    """A smooth stretching of every open axis (steps varying by a factor of
    about 1.6 along it) on the 3D reaction-diffusion workload."""
    w = _round(wl.reaction_diffusion_2d(batch=2, n=(8, 16, 16)))
    w.geom = dict(w.geom, periodic=(False, False, False))
    w.omega = _r32(np.random.default_rng(3).normal(size=w.omega.shape))
    steps = _stretched_steps(w)
    s = _solver(w)
    s.set_steps([_dev(h) for h in steps])
    z = s.forward(_dev(w.fields), _dev(w.scalars), _dev(w.rhs), _dev(w.omega)).cpu().numpy()
    for b in range(w.batch):
        zr = _oracle(w, steps, b)[4]
        assert _rel(z[b].ravel(), zr) <= FWD_TOL, (b, _rel(z[b].ravel(), zr))


def test_equal_steps_reproduce_the_uniform_solver():
    """Every interval equal to the uniform step: the same solution as the
    uniform-step solver (two different kernel paths, one system)."""
    from paper_2502_18377_b300.binding import Solver
    w = _round(_no_utt(wl.random_problem(45, (8, 16, 12), (False, True, False), batch=2)))
    steps = [_r32(np.broadcast_to(h[None, :], (w.batch, h.size))) for h in nu.uniform_intervals(w.geom)]
    args = (_dev(w.fields), _dev(w.scalars), _dev(w.rhs), _dev(w.omega))
    s = _solver(w)
    s.set_steps([_dev(h) for h in steps])
    zv = s.forward(*args).cpu().numpy()
    zu = Solver(w.geom, w.batch, w.field_of, w.fields.shape[0], max_refine=60).forward(*args).cpu().numpy()
    for b in range(w.batch):
        assert _rel(zv[b].ravel(), zu[b].ravel()) <= FWD_TOL


def test_reduced_operator_matches_oracle_schur():
    """S u (FP32 general kernels with step records) against the oracle's
    Schur complement of A^T A on unequal steps."""
    for k, w in enumerate((wl.random_problem(46, (9, 20), (False, True), batch=2),
                           wl.random_problem(47, (6, 10, 12), (False, False, True), batch=2,
                                             final_time_rows=True))):
        w = _round(w)
        steps = _steps(200 + k, w, 0.35)
        u = np.random.default_rng(0).normal(size=(w.batch, w.npoints)).astype(np.float32)
        s = _solver(w)
        s.set_steps([_dev(h) for h in steps])
        q = s.apply_reduced(_dev(w.fields), _dev(w.scalars), _dev(u)).cpu().numpy()
        for b in range(w.batch):
            el = _oracle(w, steps, b)[6]
            ref = el.S @ u[b].astype(np.float64)
            assert _rel(q[b], ref) <= 2e-5, (k, _rel(q[b], ref))


def test_steps_are_checked():
    """Missing, non-positive or non-finite steps are refused with
    INVALID_ARG, and the problem keeps no steps after a refusal."""
    from paper_2502_18377_b300.binding import MpnError
    w = _round(_no_utt(wl.random_problem(48, (6, 8), (False, True), batch=2)))
    s = _solver(w)
    args = (_dev(w.fields), _dev(w.scalars), _dev(w.rhs), _dev(w.omega))
    with pytest.raises(MpnError) as e:
        s.forward(*args)
    assert e.value.status == 1
    good = _steps(1, w, 0.2)
    for bad_value in (0.0, -0.1, float("nan"), float("inf")):
        bad = [h.copy() for h in good]
        bad[1][1, 3] = bad_value
        with pytest.raises(MpnError) as e:
            s.set_steps([_dev(h) for h in bad])
        assert e.value.status == 1
        with pytest.raises(MpnError):
            s.forward(*args)
    s.set_steps([_dev(h) for h in good])
    s.forward(*args)
    with pytest.raises(ValueError):
        s.set_steps([_dev(good[0])])
