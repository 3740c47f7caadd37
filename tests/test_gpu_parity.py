"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Both sides receive the same float32-rounded seeded inputs.  Tolerances:
  * forward z and adjoint d_z: relative L2 error <= 1e-6 per instance, on the
    whole z and on the u block (the solver's accuracy target);
  * gradients: relative L2 <= 1e-5 (they are formed from the FP32 z);
  * reduced operator apply (FP32): relative L2 <= 2e-5.
"""
import math

import numpy as np
import pytest
import torch

from oracle import assemble as asm
from oracle import grad as og
from oracle import solve as osv
from paper_2502_18377_b300 import workloads as wl

pytestmark = pytest.mark.gpu

FWD_TOL = 1e-6
GRAD_TOL = 1e-5


def _round(w):
    """float32-rounded copy of a workload (what the GPU path receives)."""
    r = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)
    return wl.Workload(w.name, w.geom, list(w.field_of), r(w.scalars), r(w.fields), r(w.rhs),
                       r(w.omega), None if w.target is None else r(w.target))


def _dev(a):
    return torch.tensor(np.asarray(a, dtype=np.float32), device="cuda").contiguous()


def _solver(w, **kw):
    from paper_2502_18377_b300.binding import Solver
    kw.setdefault("max_refine", 60)
    return Solver(w.geom, w.batch, w.field_of, w.fields.shape[0], **kw)


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _oracle_instance(w, b):
    c = w.full_coeff()[:, b]
    A, d, kind, owner = asm.assemble(w.geom, c, w.rhs[b], w.omega[b])
    z, lam, el = osv.solve_lsq_elim(A, d, asm.n_vars(w.ndim))
    return A, d, kind, owner, z, lam, el


def _no_utt(w):
    """Rough random coefficients without a u_tt term (a white-noise,
    random-sign second time derivative makes the problem mixed-type, where
    the solver converges but slowly)."""
    w.fields[2] = 0.0
    return w


def _rd_fields(w, layout):
    """Reaction-diffusion with another assignment of its coefficient fields
    (c_0, c_xx, c_yy stay fields, the fused step's compile-time layout):
    "three" gives c_yy a field of its own (anisotropic diffusion), "one"
    makes c_0, c_xx and c_yy one field."""
    if layout == "three":
        d2 = w.fields[0] * (1.0 + 0.5 * np.cos(np.linspace(0.0, 3.0, w.npoints)))[None, :]
        fields = np.concatenate([w.fields, d2[None]], axis=0)
        field_of = [1, -1, -1, -1, 0, -1, 2]
    else:
        fields = w.fields[:1].copy()
        field_of = [0, -1, -1, -1, 0, -1, 0]
    return wl.Workload(w.name + "_" + layout, w.geom, field_of, w.scalars, fields, w.rhs, w.omega, w.target)


CASES = [
    ("c1_full", lambda: wl.advection_diffusion_1d()),
    ("c2_small", lambda: wl.reaction_diffusion_2d(batch=3, n=(8, 16, 16))),
    ("c2_ragged", lambda: wl.reaction_diffusion_2d(batch=2, n=(10, 12, 20))),
    # the fused step's compile-time layout with three distinct fields on
    # 4-plane tiles, with one field, and with 128-point y rows
    ("c2_three_fields", lambda: _rd_fields(wl.reaction_diffusion_2d(batch=2, n=(12, 16, 32)), "three")),
    ("c2_one_field", lambda: _rd_fields(wl.reaction_diffusion_2d(batch=2, n=(8, 16, 16)), "one")),
    ("c2_wide_y", lambda: wl.reaction_diffusion_2d(batch=1, n=(8, 8, 128))),
    ("c3_small", lambda: wl.linearized_burgers_1d(batch=2, n=(32, 64))),
    ("c5_small", lambda: wl.transport_2d(batch=2, n=(8, 16, 16))),
    ("rand_dirichlet_2d", lambda: _no_utt(wl.random_problem(21, (12, 32), (False, False), batch=2))),
    ("rand_odd_2d_final", lambda: wl.random_problem(22, (9, 13), (False, False), batch=2,
                                                    final_time_rows=True)),
    ("rand_mixed_3d", lambda: _no_utt(wl.random_problem(23, (7, 16, 12), (False, True, False), batch=2))),
    ("rand_utt_2d", lambda: wl.random_problem(25, (10, 16), (False, True), batch=2)),
    ("rand_scalars_3d", lambda: wl.random_problem(24, (6, 8, 8), (False, True, True), batch=3,
                                                  field_all=False)),
    # float4 levels run the fused operator step; these two put Dirichlet x and
    # y faces, one-sided edge rows and final-time rows inside its tiles
    ("rand_dirichlet_3d", lambda: _no_utt(wl.random_problem(26, (8, 16, 12), (False, False, False), batch=2))),
    ("rand_final_3d", lambda: _no_utt(wl.random_problem(27, (12, 8, 16), (False, False, True), batch=2,
                                                        final_time_rows=True))),
    # 1-D + t float4 groups: Dirichlet x faces inside the groups, final-time rows
    ("rand_final_2d", lambda: _no_utt(wl.random_problem(28, (9, 16), (False, False), batch=2,
                                                        final_time_rows=True))),
    # Laplace's equation (elliptic in both axes, Dirichlet on all four faces)
    ("laplace_32", lambda: wl.laplace_2d(batch=2, n=32)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_forward_matches_oracle(name, make):
    w = _round(make())
    s = _solver(w)
    z = s.forward(_dev(w.fields), _dev(w.scalars), _dev(w.rhs), _dev(w.omega)).cpu().numpy()
    V, N = asm.n_vars(w.ndim), w.npoints
    for b in range(w.batch):
        zr = _oracle_instance(w, b)[4]
        assert _rel(z[b].ravel(), zr) <= FWD_TOL, (name, b, _rel(z[b].ravel(), zr), s.last_stats)
        assert _rel(z[b, 0], zr[:N]) <= FWD_TOL


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_forward_passwise_levels_match_oracle(name, make):
    """The same solve with every operator pass a kernel of its own (no fused
    coarse end, no fused operator step): both schedules meet the oracle, and
    the fused coarse end is in use by default wherever two or more levels
    fit."""
    w = _round(make())
    s = _solver(w, fused_coarse=False, fused_step=False)
    assert s.fused_level() == -1
    z = s.forward(_dev(w.fields), _dev(w.scalars), _dev(w.rhs), _dev(w.omega)).cpu().numpy()
    for b in range(w.batch):
        zr = _oracle_instance(w, b)[4]
        assert _rel(z[b].ravel(), zr) <= FWD_TOL, (name, b, _rel(z[b].ravel(), zr), s.last_stats)
    sf = _solver(w)
    if len(sf.levels()) >= 2:
        assert sf.fused_level() >= 0, sf.levels()
    zf = sf.forward(_dev(w.fields), _dev(w.scalars), _dev(w.rhs), _dev(w.omega)).cpu().numpy()
    # both schedules apply the same preconditioner up to FP32 rounding order;
    # where PCG needs hundreds of iterations (the mixed-type u_tt case) that
    # rounding changes the count, so the counts are compared only below 100
    it_f, it_p = sf.last_stats["pcg_iters"], s.last_stats["pcg_iters"]
    if it_p < 100:
        assert abs(it_f - it_p) <= 6, (sf.last_stats, s.last_stats)
    assert _rel(zf.ravel(), z.ravel()) <= 2 * FWD_TOL


DIRECT_CASES = ["c1_full", "c3_small", "rand_dirichlet_2d", "rand_odd_2d_final", "rand_utt_2d",
                "rand_scalars_3d", "laplace_32"]


@pytest.mark.parametrize("name,make", [c for c in CASES if c[0] in DIRECT_CASES],
                         ids=[c[0] for c in CASES if c[0] in DIRECT_CASES])
def test_direct_path_matches_oracle(name, make):
    """Small problems through the direct path (no hierarchy; the reduced
    system's banded Cholesky factor and explicit inverse, in shared or global
    memory by band size): forward and adjoint meet the oracle."""
    w = _round(make())
    s = _solver(w, direct=True)
    assert len(s.levels()) == 1
    args = (_dev(w.fields), _dev(w.scalars), _dev(w.rhs), _dev(w.omega))
    z = s.forward(*args)
    zc = z.cpu().numpy()
    rng = np.random.default_rng(7)
    V, N = asm.n_vars(w.ndim), w.npoints
    g = rng.normal(size=(w.batch, V, N)).astype(np.float32)
    _, _, drhs, _, dz = s.adjoint(*args, z, _dev(g), reuse_setup=True, want_dz=True)
    dz = dz.cpu().numpy()
    for b in range(w.batch):
        A, d, kind, owner, zr, lam, el = _oracle_instance(w, b)
        assert _rel(zc[b].ravel(), zr) <= FWD_TOL, (name, b, _rel(zc[b].ravel(), zr), s.last_stats)
        dzr, _ = og.adjoint_elim(el, g[b].astype(np.float64).ravel())
        assert _rel(dz[b].ravel(), dzr) <= FWD_TOL, (name, b, _rel(dz[b].ravel(), dzr))


def test_direct_path_rejects_wide_bands():
    from paper_2502_18377_b300.binding import MpnError
    w = wl.reaction_diffusion_2d(batch=1, n=(8, 16, 16))      # band 3 * 256 - 1 >= 256
    with pytest.raises(MpnError) as e:
        _solver(w, direct=True)
    assert e.value.status == 2


@pytest.mark.parametrize("krylov", ["cg", "fgmres"])
def test_laplace_with_time_axis_coarsened_matches_oracle(krylov):
    """Laplace's equation is elliptic in the first axis as well: the hierarchy
    that halves it too (coarsen_time) reaches the oracle's solution."""
    w = _round(wl.laplace_2d(batch=2, n=32))
    s = _solver(w, coarsen_time=True, krylov=krylov)
    assert s.levels()[1][0] == 16, s.levels()
    z = s.forward(_dev(w.fields), _dev(w.scalars), _dev(w.rhs), _dev(w.omega)).cpu().numpy()
    for b in range(w.batch):
        zr = _oracle_instance(w, b)[4]
        assert _rel(z[b].ravel(), zr) <= FWD_TOL, (b, _rel(z[b].ravel(), zr), s.last_stats)


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_fgmres_forward_and_adjoint_match_oracle(name, make):
    """The refinement with flexible GMRES (Section 3.1's solver) as the inner
    FP32 solve instead of CG meets the same tolerances."""
    w = _round(make())
    s = _solver(w, krylov="fgmres")
    args = (_dev(w.fields), _dev(w.scalars), _dev(w.rhs), _dev(w.omega))
    z = s.forward(*args)
    zc = z.cpu().numpy()
    rng = np.random.default_rng(6)
    V, N = asm.n_vars(w.ndim), w.npoints
    g = rng.normal(size=(w.batch, V, N)).astype(np.float32)
    _, _, drhs, _, dz = s.adjoint(*args, z, _dev(g), reuse_setup=True, want_dz=True)
    dz, drhs = dz.cpu().numpy(), drhs.cpu().numpy()
    for b in range(w.batch):
        A, d, kind, owner, zr, lam, el = _oracle_instance(w, b)
        assert _rel(zc[b].ravel(), zr) <= FWD_TOL, (name, b, _rel(zc[b].ravel(), zr), s.last_stats)
        dzr, dlamr = og.adjoint_elim(el, g[b].astype(np.float64).ravel())
        assert _rel(dz[b].ravel(), dzr) <= FWD_TOL, (name, b, _rel(dz[b].ravel(), dzr))


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_adjoint_and_gradients_match_oracle(name, make):
    w = _round(make())
    s = _solver(w)
    F = w.fields.shape[0]
    args = (_dev(w.fields), _dev(w.scalars), _dev(w.rhs), _dev(w.omega))
    z = s.forward(*args)
    rng = np.random.default_rng(5)
    V, N = asm.n_vars(w.ndim), w.npoints
    g = rng.normal(size=(w.batch, V, N)).astype(np.float32)
    dfields, dscal, drhs, dom, dz = s.adjoint(*args, z, _dev(g), reuse_setup=True, want_dz=True)
    dfields, dscal, drhs, dom, dz = (t.cpu().numpy() for t in (dfields, dscal, drhs, dom, dz))
    zc = z.cpu().numpy()
    for b in range(w.batch):
        A, d, kind, owner, zr, lam, el = _oracle_instance(w, b)
        dzr, dlamr = og.adjoint_elim(el, g[b].astype(np.float64).ravel())
        assert _rel(dz[b].ravel(), dzr) <= FWD_TOL, (name, b, _rel(dz[b].ravel(), dzr))
        dc, db, dw = og.gradients(w.geom, A, d, kind, owner, zr, lam, dzr, dlamr)
        for f in range(F):
            ref = sum(dc[v] for v in range(V) if w.field_of[v] == f)
            assert _rel(dfields[f, b], ref) <= GRAD_TOL, (name, "field", f, _rel(dfields[f, b], ref))
        for v in range(V):
            if w.field_of[v] < 0:
                assert abs(dscal[v, b] - dc[v].sum()) <= GRAD_TOL * max(1.0, np.abs(dc[v]).sum())
        assert _rel(drhs[b], db) <= GRAD_TOL
        assert _rel(dom[b], dw) <= GRAD_TOL


def test_reduced_operator_matches_oracle_schur():
    """S u (FP32 kernels) against the oracle's Schur complement of A^T A."""
    for w in (wl.random_problem(31, (9, 20), (False, True), batch=2),
              # 1-D + t float4 groups with Dirichlet x faces and final-time rows
              wl.random_problem(34, (10, 24), (False, False), batch=2, final_time_rows=True),
              wl.random_problem(32, (6, 10, 12), (False, False, True), batch=2, final_time_rows=True),
              _round(wl.reaction_diffusion_2d(batch=2, n=(8, 16, 16))),
              wl.random_problem(33, (8, 12, 16), (False, False, False), batch=2, final_time_rows=True)):
        w = _round(w)
        rng = np.random.default_rng(0)
        u = rng.normal(size=(w.batch, w.npoints)).astype(np.float32)
        # the last two run the fused operator step at the finest level
        for fused in (True, False):
            s = _solver(w, fused_step=fused)
            q = s.apply_reduced(_dev(w.fields), _dev(w.scalars), _dev(u)).cpu().numpy()
            for b in range(w.batch):
                A, d, kind, owner, zr, lam, el = _oracle_instance(w, b)
                ref = el.S @ u[b].astype(np.float64)
                assert _rel(q[b], ref) <= 2e-5, (fused, _rel(q[b], ref))


def test_forward_is_deterministic():
    w = _round(wl.reaction_diffusion_2d(batch=2, n=(8, 16, 16)))
    s = _solver(w)
    args = (_dev(w.fields), _dev(w.scalars), _dev(w.rhs), _dev(w.omega))
    z1 = s.forward(*args).cpu().numpy()
    z2 = s.forward(*args).cpu().numpy()
    assert np.array_equal(z1, z2)


def test_one_problem_solves_new_coefficients_each_call():
    """The setup after the input copies is captured once and replayed: a
    problem object given other coefficients, right-hand sides and boundary
    data (another seed; then the first data again) must solve each set, in
    both directions, to the oracle's tolerance."""
    wa = _round(wl.reaction_diffusion_2d(batch=2, n=(8, 16, 16), seed_base=2000))
    wb = _round(wl.reaction_diffusion_2d(batch=2, n=(8, 16, 16), seed_base=7000))
    assert not np.allclose(wa.fields, wb.fields)
    s = _solver(wa)
    V, N = asm.n_vars(wa.ndim), wa.npoints
    rng = np.random.default_rng(9)
    g = rng.normal(size=(wa.batch, V, N)).astype(np.float32)
    for w in (wa, wb, wa):
        args = (_dev(w.fields), _dev(w.scalars), _dev(w.rhs), _dev(w.omega))
        z = s.forward(*args)
        _, _, _, _, dz = s.adjoint(*args, z, _dev(g), reuse_setup=True, want_dz=True)
        z, dz = z.cpu().numpy(), dz.cpu().numpy()
        for b in range(w.batch):
            A, d, kind, owner, zr, lam, el = _oracle_instance(w, b)
            assert _rel(z[b].ravel(), zr) <= FWD_TOL, (b, _rel(z[b].ravel(), zr))
            dzr, _ = og.adjoint_elim(el, g[b].astype(np.float64).ravel())
            assert _rel(dz[b].ravel(), dzr) <= FWD_TOL, (b, _rel(dz[b].ravel(), dzr))


@pytest.mark.parametrize("cheb_degree,inner_iters,adj_inner_iters",
                         [(1, 5, 0), (2, 5, 0), (5, 1, 0), (3, 2, 0), (5, 5, 9), (3, 7, 2)])
def test_smoother_degree_and_inner_iterations_meet_the_oracle(cheb_degree, inner_iters, adj_inner_iters):
    """The finest level's folded steps depend on the schedule: with degree 1
    the V-cycle has no Chebyshev post-smoothing step to sum <z, r> (z is
    copied out), one PCG iteration per sweep never updates the direction, and
    short smoothers change which buffer each step reads; the adjoint may run
    its own count per sweep.  Every combination meets the oracle in both
    directions."""
    w = _round(wl.reaction_diffusion_2d(batch=2, n=(8, 16, 16)))
    s = _solver(w, cheb_degree=cheb_degree, inner_iters=inner_iters, adj_inner_iters=adj_inner_iters)
    V, N = asm.n_vars(w.ndim), w.npoints
    g = np.random.default_rng(11).normal(size=(w.batch, V, N)).astype(np.float32)
    args = (_dev(w.fields), _dev(w.scalars), _dev(w.rhs), _dev(w.omega))
    z = s.forward(*args)
    _, _, _, _, dz = s.adjoint(*args, z, _dev(g), reuse_setup=True, want_dz=True)
    if adj_inner_iters:
        assert s.last_stats["pcg_iters"] % adj_inner_iters == 0, s.last_stats   # sweeps of the adjoint's count
    z, dz = z.cpu().numpy(), dz.cpu().numpy()
    for b in range(w.batch):
        A, d, kind, owner, zr, lam, el = _oracle_instance(w, b)
        assert _rel(z[b].ravel(), zr) <= FWD_TOL, (b, _rel(z[b].ravel(), zr), s.last_stats)
        dzr, _ = og.adjoint_elim(el, g[b].astype(np.float64).ravel())
        assert _rel(dz[b].ravel(), dzr) <= FWD_TOL, (b, _rel(dz[b].ravel(), dzr))


def test_gradients_match_finite_differences_burgers():
    """Linearized Burgers, L = mean((u - target)^2): dL/dc, dL/df and dL/du0
    from the adjoint kernels against central differences of the FP64 oracle
    at 20 random coordinates (relative 1e-3)."""
    w = _round(wl.linearized_burgers_1d(batch=1, n=(16, 32)))
    N = w.npoints
    s = _solver(w)
    args = [_dev(w.fields), _dev(w.scalars), _dev(w.rhs), _dev(w.omega)]
    z = s.forward(*args)
    tgt = _dev(w.target)
    gz = s.mse_grad(z, tgt)
    dfields, dscal, drhs, dom = s.adjoint(*args, z, gz, reuse_setup=True)
    dfields, drhs, dom = dfields.cpu().numpy()[0, 0], drhs.cpu().numpy()[0], dom.cpu().numpy()[0]

    def loss(fields, rhs, omega):
        ww = wl.Workload(w.name, w.geom, w.field_of, w.scalars, fields, rhs, omega)
        A, d, *_ = asm.assemble(w.geom, ww.full_coeff()[:, 0], rhs[0], omega[0])
        zz, _, _ = osv.solve_lsq_elim(A, d, 5)
        return float(((zz[:N] - w.target[0]) ** 2).mean())

    rng = np.random.default_rng(3)
    h = 1e-4
    checked = 0
    for k in range(20):
        kind = k % 3
        if kind == 0:
            p = rng.integers(0, N)
            fp, fm = w.fields.copy(), w.fields.copy()
            fp[0, 0, p] += h; fm[0, 0, p] -= h
            fd = (loss(fp, w.rhs, w.omega) - loss(fm, w.rhs, w.omega)) / (2 * h)
            an = dfields[p]
        elif kind == 1:
            p = rng.integers(0, N)
            rp, rm = w.rhs.copy(), w.rhs.copy()
            rp[0, p] += h; rm[0, p] -= h
            fd = (loss(w.fields, rp, w.omega) - loss(w.fields, rm, w.omega)) / (2 * h)
            an = drhs[p]
        else:
            p = rng.integers(0, w.geom["n"][1])   # a point of the t = 0 face
            op, om = w.omega.copy(), w.omega.copy()
            op[0, p] += h; om[0, p] -= h
            fd = (loss(w.fields, w.rhs, op) - loss(w.fields, w.rhs, om)) / (2 * h)
            an = dom[p]
        scale = max(abs(fd), 1e-3 * max(np.abs(dfields).max(), np.abs(drhs).max(), np.abs(dom).max()))
        assert abs(an - fd) <= 1e-3 * scale, (k, kind, an, fd)
        checked += 1
    assert checked == 20


def test_error_statuses_without_a_gpu_fault():
    """Failure handling is host-visible status, never a device fault: NaN in
    the inputs -> NONFINITE, too few refinement sweeps -> NOT_CONVERGED with
    the statistics written, and the problem stays usable afterwards."""
    from paper_2502_18377_b300.binding import MpnError
    w = _round(wl.reaction_diffusion_2d(batch=2, n=(8, 16, 16)))
    s = _solver(w)
    args = [_dev(w.fields), _dev(w.scalars), _dev(w.rhs), _dev(w.omega)]
    bad = args[2].clone()
    bad[1, 17] = float("nan")
    with pytest.raises(MpnError) as e:
        s.forward(args[0], args[1], bad, args[3])
    assert e.value.status == 4, e.value
    s1 = _solver(w, max_refine=1)
    with pytest.raises(MpnError) as e:
        s1.forward(*args)
    assert e.value.status == 3
    assert s1.last_stats["sweeps"] == 1 and s1.last_stats["pcg_iters"] > 0
    z = s1.forward(*args, allow_not_converged=True)
    assert torch.isfinite(z).all()
    # the first problem still solves correctly after the failed call
    z = s.forward(*args).cpu().numpy()
    zr = _oracle_instance(w, 0)[4]
    assert _rel(z[0].ravel(), zr) <= FWD_TOL


YSPLIT_CASES = [
    # transport (c_x, c_y fields: its compile-time layout), 2 y segments
    ("transport_tr", lambda: wl.transport_2d(batch=2, n=(8, 8, 128))),
    # reaction-diffusion (c_0, c_xx = c_yy fields)
    ("reaction_diffusion_rdi", lambda: wl.reaction_diffusion_2d(batch=2, n=(8, 8, 128))),
    # run-time layouts with Dirichlet y faces (one-sided rows inside the
    # first and last segment), Dirichlet x, final-time rows
    ("rand_dirichlet_y", lambda: _no_utt(wl.random_problem(71, (8, 8, 128), (False, True, False), batch=2))),
    ("rand_dirichlet_xy_final", lambda: _no_utt(wl.random_problem(72, (8, 8, 128), (False, False, False), batch=1,
                                                                  final_time_rows=True))),
    ("rand_periodic_xy", lambda: _no_utt(wl.random_problem(73, (8, 12, 128), (False, True, True), batch=2))),
]


@pytest.mark.parametrize("name,make", YSPLIT_CASES, ids=[c[0] for c in YSPLIT_CASES])
def test_ysplit_tiles_match_oracle(name, make):
    """The fused step on tiles of 64-point y segments (fused_step = 2 puts
    it on every level with rows of >= 128 points): the reduced operator, the
    forward solve and the adjoint solve meet the oracle at the tolerances of
    the whole-row schedule."""
    w = _round(make())
    s = _solver(w, fused_step=2)
    rng = np.random.default_rng(74)
    V, N = asm.n_vars(w.ndim), w.npoints
    u = rng.normal(size=(w.batch, N)).astype(np.float32)
    q = s.apply_reduced(_dev(w.fields), _dev(w.scalars), _dev(u)).cpu().numpy()
    args = (_dev(w.fields), _dev(w.scalars), _dev(w.rhs), _dev(w.omega))
    z = s.forward(*args)
    g = rng.normal(size=(w.batch, V, N)).astype(np.float32)
    _, _, _, _, dz = s.adjoint(*args, z, _dev(g), reuse_setup=True, want_dz=True)
    z, dz = z.cpu().numpy(), dz.cpu().numpy()
    for b in range(w.batch):
        A, d, kind, owner, zr, lam, el = _oracle_instance(w, b)
        ref = el.S @ u[b].astype(np.float64)
        assert _rel(q[b], ref) <= 2e-5, (name, b, _rel(q[b], ref))
        assert _rel(z[b].ravel(), zr) <= FWD_TOL, (name, b, _rel(z[b].ravel(), zr), s.last_stats)
        dzr, _ = og.adjoint_elim(el, g[b].astype(np.float64).ravel())
        assert _rel(dz[b].ravel(), dzr) <= FWD_TOL, (name, b, _rel(dz[b].ravel(), dzr))


def test_ysplit_operator_three_segments():
    """Rows of 192 points: three 64-point y segments, the middle one with y
    halos inside the domain on both sides, with Dirichlet and periodic y.
    (The solve is not run: with white-noise coefficients the hierarchy that
    halves y five times but x once converges too slowly on this shape, with
    either schedule.)"""
    for per in ((False, False, False), (False, True, True), (False, False, True)):
        w = _round(_no_utt(wl.random_problem(75, (8, 8, 192), per, batch=2, final_time_rows=not per[2])))
        u = np.random.default_rng(76).normal(size=(w.batch, w.npoints)).astype(np.float32)
        s = _solver(w, fused_step=2)
        q = s.apply_reduced(_dev(w.fields), _dev(w.scalars), _dev(u)).cpu().numpy()
        for b in range(w.batch):
            el = _oracle_instance(w, b)[6]
            ref = el.S @ u[b].astype(np.float64)
            assert _rel(q[b], ref) <= 2e-5, (per, b, _rel(q[b], ref))


def test_device_error_word_reaches_the_host():
    """The error word a kernel's bounded wait sets when it gives up is read
    back with each sweep's scalars and turned into MPN_ERR_CUDA.  Injected on
    the host (no kernel waits or faults); the next solve starts with the word
    clear and meets the oracle."""
    from paper_2502_18377_b300.binding import MpnError
    w = _round(wl.reaction_diffusion_2d(batch=2, n=(8, 16, 16)))
    s = _solver(w)
    args = [_dev(w.fields), _dev(w.scalars), _dev(w.rhs), _dev(w.omega)]
    s.inject_wait_failure()
    with pytest.raises(MpnError) as e:
        s.forward(*args)
    assert e.value.status == 6 and "bounded wait" in str(e.value), e.value
    z = s.forward(*args).cpu().numpy()
    zr = _oracle_instance(w, 0)[4]
    assert _rel(z[0].ravel(), zr) <= FWD_TOL
