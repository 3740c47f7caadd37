"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each checks it against a
number the paper prints, a closed form, a textbook/library routine on a tiny
case, or an invariant, chosen so that a dropped term, a wrong sign, a wrong
index or a transposed operand in the oracle fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
import torch

from oracle import assemble as asm
from oracle import grad as og
from oracle import solve as osv
from paper_2502_18377_b300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _geom(n, periodic, stencil=3, final=False, lengths=None):
    lengths = lengths or (1.0,) * len(n)
    step = tuple(L / k if p else L / (k - 1) for k, p, L in zip(n, periodic, lengths))
    return dict(n=tuple(n), step=step, periodic=tuple(periodic), stencil=stencil,
                final_time_rows=final)


# ---------------------------------------------------------------- row counts
def test_counts_match_paper_32x32():
    """Section 3 'Scaling PDE Solving': 5120 variables, 9212 constraints and
    377 MB of dense FP64 storage for a 32x32 grid, > 99.9% zeros."""
    ref = json.load(open(os.path.join(GOLDEN, "paper_counts.json")))
    g = _geom((32, 32), (False, False), final=True)
    A, d, kind, owner = asm.assemble(g, np.ones((5, 1024)), np.zeros(1024), np.zeros(1024))
    assert A.shape == (ref["grid_32x32"]["constraints"], ref["grid_32x32"]["variables"])
    assert round(A.shape[0] * A.shape[1] * 8 / 1e6) == ref["grid_32x32"]["dense_fp64_MB"]
    assert 1.0 - A.nnz / (A.shape[0] * A.shape[1]) > ref["sparsity_32x32_min"]
    assert asm.counts(g) == (A.shape[1], A.shape[0])


def test_counts_match_paper_3d():
    """Same paragraph: ~220k variables / ~420k constraints / 780 GB for 32^3,
    50k GB for 64^3, 99.999% zeros for 64^3."""
    ref = json.load(open(os.path.join(GOLDEN, "paper_counts.json")))
    g = _geom((32, 32, 32), (False,) * 3, final=True)
    nv, nc = asm.counts(g)
    r = ref["grid_32x32x32"]
    assert abs(nv - r["variables_approx"]) / r["variables_approx"] < 0.05
    assert abs(nc - r["constraints_approx"]) / r["constraints_approx"] < 0.05
    assert round(nv * nc * 8 / 1e9, -1) == r["dense_fp64_GB"]
    A, *_ = asm.assemble(g, np.ones((7, 32768)), np.zeros(32768), np.zeros(32768))
    assert A.shape == (nc, nv)
    g64 = _geom((64, 64, 64), (False,) * 3, final=True)
    nv, nc = asm.counts(g64)
    assert round(nv * nc * 8 / 1e9, -3) == ref["grid_64x64x64"]["dense_fp64_GB"]
    A, *_ = asm.assemble(g64, np.ones((7, 64 ** 3)), np.zeros(64 ** 3), np.zeros(64 ** 3))
    assert A.shape == (nc, nv)
    assert 1.0 - A.nnz / (A.shape[0] * A.shape[1]) > ref["sparsity_64x64x64_min"]


@pytest.mark.parametrize("n,per,st", [((8, 6), (False, True), 3), ((7, 9), (False, False), 5),
                                      ((5, 6, 7), (False, True, False), 3),
                                      ((6, 5, 8), (False, True, True), 5)])
def test_count_formula_matches_assembly(n, per, st):
    g = _geom(n, per, st)
    N = int(np.prod(n))
    A, *_ = asm.assemble(g, np.ones((asm.n_vars(len(n)), N)), np.zeros(N), np.zeros(N))
    assert asm.counts(g) == (A.shape[1], A.shape[0])


# ------------------------------------------------------ closed-form solutions
def _exact_factor(rng, k, s, periodic):
    """One-dimensional factor g with values and the derivative values that make
    every row along this dimension exact.

    Non-periodic: a random quadratic; Taylor rows (Eqs. 6-7), central and
    one-sided difference rows are exact for quadratics.
    Periodic: the real discrete Fourier mode cos(theta j + phi); its exact
    three-point symbols are s u' = -sin(theta) sin(theta j + phi) and
    s^2 u'' = 2 (cos(theta) - 1) cos(theta j + phi), with which the Taylor rows
    hold exactly too (cos(theta j + phi +- theta) expanded)."""
    j = np.arange(k)
    if not periodic:
        a0, a1, a2 = rng.normal(size=3)
        x = j * s
        return a0 + a1 * x + a2 * x * x, a1 + 2 * a2 * x, np.full(k, 2 * a2)
    th = 2 * math.pi * rng.integers(1, max(2, k // 2)) / k
    ph = rng.uniform(0, 2 * math.pi)
    return (np.cos(th * j + ph), -math.sin(th) * np.sin(th * j + ph) / s,
            2 * (math.cos(th) - 1) * np.cos(th * j + ph) / s ** 2)


def _exact_solution(rng, g):
    """z with A z = d exactly for a separable u = prod_d g_d(x_d)."""
    n = g["n"]
    D = len(n)
    fac = [_exact_factor(rng, n[d], g["step"][d], g["periodic"][d]) for d in range(D)]
    V = asm.n_vars(D)

    def outer(parts):
        out = parts[0]
        for p in parts[1:]:
            out = np.multiply.outer(out, p)
        return out.ravel()

    z = np.empty((V, int(np.prod(n))))
    z[0] = outer([f[0] for f in fac])
    for d in range(D):
        for kk, var in ((1, asm.first(d)), (2, asm.second(d))):
            z[var] = outer([fac[e][kk] if e == d else fac[e][0] for e in range(D)])
    return z


@pytest.mark.parametrize("n,per,st", [((6, 7), (False, False), 3), ((6, 8), (False, True), 3),
                                      ((7, 9), (False, False), 5),
                                      ((5, 6, 8), (False, True, True), 3),
                                      ((6, 5, 7), (False, False, False), 5),
                                      ((5, 8, 6), (False, True, False), 3)])
def test_closed_form_zero_residual_and_recovered(n, per, st):
    """With b = sum_v c_v z_v (random c fields) and omega = u, the exact z has
    zero residual, so the least-squares solution must be that z."""
    rng = np.random.default_rng(7)
    g = _geom(n, per, st)
    N = int(np.prod(n))
    V = asm.n_vars(len(n))
    z = _exact_solution(rng, g)
    c = rng.uniform(-1, 1, size=(V, N))
    b = (c * z).sum(0)
    A, d, kind, owner = asm.assemble(g, c, b, z[0])
    assert np.abs(A @ z.ravel() - d).max() < 1e-9 * max(1.0, np.abs(z).max())
    zs, lam, _ = osv.solve_lsq(A, d)
    assert np.linalg.norm(zs - z.ravel()) <= 1e-8 * np.linalg.norm(z)
    assert np.abs(lam).max() < 1e-8


@pytest.mark.parametrize("n,per,st,orders", [
    ((0, 0), (False, True), 3, {asm.D1: 3, asm.D2: 4, asm.TF: 3, asm.TB: 3}),
    ((0, 0), (False, True), 5, {asm.D1: 5, asm.D2: 6, asm.TF: 3, asm.TB: 3}),
])
def test_consistency_order_periodic(n, per, st, orders):
    """Rows evaluated on an analytic periodic u(t, x) = exp(-t) sin(2 pi x)
    with its exact derivatives: the residual of each family falls as s^(p + k),
    p the order of its difference formula and k the s-power its row carries
    (central first/second differences: 2 + 1 / 2 + 2 for three points,
    4 + 1 / 4 + 2 for five; Taylor rows drop the third-order term: 3).  Time
    rows are evaluated only away from the t-edges."""
    errs = {k: [] for k in orders}
    for m in (32, 64, 128):
        g = _geom((m, m), per, st)
        t = np.arange(m) * g["step"][0]
        x = np.arange(m) * g["step"][1]
        T, X = np.meshgrid(t, x, indexing="ij")
        w = 2 * math.pi
        u = np.exp(-T) * np.sin(w * X)
        z = np.stack([u, -u, u, w * np.exp(-T) * np.cos(w * X), -w * w * u]).reshape(5, -1)
        N = m * m
        c = np.ones((5, N))
        b = (c * z).sum(0)
        A, d, kind, owner = asm.assemble(g, c, b, u.ravel())
        r = A @ z.ravel() - d
        it = owner // m
        interior = (it >= 2) & (it <= m - 3)
        for fam in orders:
            sel = (kind == fam) & interior
            errs[fam].append(np.abs(r[sel]).max())
        assert np.abs(r[(kind == asm.E) | (kind == asm.BC)]).max() < 1e-12
    for fam, p in orders.items():
        e = errs[fam]
        rate = math.log2(e[1] / e[2])
        assert rate > p - 0.3, (fam, e, rate)


def test_heat_mode_convergence():
    """u = exp(-nu k^2 t) sin(k x) solves u_t - nu u_xx = 0 (periodic x): the
    least-squares solution approaches it as the grid refines."""
    nu, k = 0.05, 2 * math.pi
    errs = []
    for m in (16, 32, 64):
        g = _geom((m, m), (False, True))
        t = np.arange(m) * g["step"][0]
        x = np.arange(m) * g["step"][1]
        T, X = np.meshgrid(t, x, indexing="ij")
        u = np.exp(-nu * k * k * T) * np.sin(k * X)
        N = m * m
        c = np.zeros((5, N)); c[1] = 1.0; c[4] = -nu
        A, d, kind, owner = asm.assemble(g, c, np.zeros(N), u.ravel())
        z, _, _ = osv.solve_lsq(A, d)
        errs.append(np.linalg.norm(z[:N] - u.ravel()) / np.linalg.norm(u))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 2e-3
    assert math.log2(errs[1] / errs[2]) > 1.5, errs


def test_advection_translation_convergence():
    """u = sin(2 pi (x - a t)) is translated exactly by u_t + a u_x = 0."""
    a = 0.7
    errs = []
    for m in (16, 32, 64):
        g = _geom((m, m), (False, True))
        t = np.arange(m) * g["step"][0]
        x = np.arange(m) * g["step"][1]
        T, X = np.meshgrid(t, x, indexing="ij")
        u = np.sin(2 * math.pi * (X - a * T))
        N = m * m
        c = np.zeros((5, N)); c[1] = 1.0; c[3] = a
        A, d, kind, owner = asm.assemble(g, c, np.zeros(N), u.ravel())
        z, _, _ = osv.solve_lsq(A, d)
        errs.append(np.linalg.norm(z[:N] - u.ravel()) / np.linalg.norm(u))
    assert errs[0] > errs[1] > errs[2]
    assert math.log2(errs[1] / errs[2]) > 1.5, errs


def test_laplace_converges_to_harmonic_solution():
    """Laplace's equation (the paper's solver unit test), with the grid's first
    axis as y, Dirichlet data on all four faces from u = sinh(pi y) sin(pi x) /
    sinh(pi) + 0.5 sinh(2 pi y) sin(2 pi x) / sinh(2 pi): the least-squares
    solution approaches this harmonic function as the grid is refined."""
    errs = []
    for m in (8, 16, 32):
        g = _geom((m, m), (False, False), final=True)
        y = np.arange(m) * g["step"][0]
        x = np.arange(m) * g["step"][1]
        Y, X = np.meshgrid(y, x, indexing="ij")
        u = (np.sinh(math.pi * Y) * np.sin(math.pi * X) / math.sinh(math.pi)
             + 0.5 * np.sinh(2 * math.pi * Y) * np.sin(2 * math.pi * X) / math.sinh(2 * math.pi))
        N = m * m
        c = np.zeros((5, N)); c[2] = 1.0; c[4] = 1.0
        A, d, kind, owner = asm.assemble(g, c, np.zeros(N), u.ravel())
        z, _, _ = osv.solve_lsq(A, d)
        errs.append(np.linalg.norm(z[:N] - u.ravel()) / np.linalg.norm(u))
    assert errs[0] > errs[1] > errs[2]
    assert errs[0] / errs[1] > 4 and errs[1] / errs[2] > 4, errs
    assert errs[2] < 5e-3, errs


# ------------------------------------------------------------- the LS solve
@pytest.mark.parametrize("n,per,st", [((6, 6), (False, False), 3), ((6, 8), (False, True), 5),
                                      ((4, 5, 6), (False, True, False), 3)])
def test_solve_matches_dense_lstsq(n, per, st):
    """Brute force: numpy's dense least squares (SVD) on the assembled matrix."""
    w = wl.random_problem(11, n, per, st)
    c = w.full_coeff()[:, 0]
    A, d, kind, owner = asm.assemble(w.geom, c, w.rhs[0], w.omega[0])
    z, lam, _ = osv.solve_lsq(A, d)
    Ad = A.toarray()
    zref = np.linalg.lstsq(Ad, d, rcond=None)[0]
    assert np.linalg.norm(z - zref) <= 1e-10 * np.linalg.norm(zref)
    assert np.linalg.matrix_rank(Ad) == Ad.shape[1]           # full column rank
    assert np.linalg.norm(lam - (d - Ad @ zref)) <= 1e-10 * np.linalg.norm(d)
    assert np.abs(Ad.T @ lam).max() < 1e-10 * np.abs(d).max()  # A^T lambda* = 0
    zn = osv.solve_normal(A, d)
    assert np.linalg.norm(zn - zref) <= 1e-8 * np.linalg.norm(zref)


def test_normal_matrix_symmetric_positive():
    w = wl.random_problem(3, (5, 6, 6), (False, True, True), 3)
    A, d, *_ = asm.assemble(w.geom, w.full_coeff()[:, 0], w.rhs[0], w.omega[0])
    M = (A.T @ A).toarray()
    assert np.abs(M - M.T).max() == 0.0
    assert np.linalg.eigvalsh(M).min() > 0


# --------------------------------------------------------------- gradients
def _loss_and_g(z, tgt, N):
    """L = mean over points of (u - target)^2 and its gradient wrt z."""
    r = z[:N] - tgt
    g = np.zeros_like(z)
    g[:N] = 2 * r / N
    return float((r * r).mean()), g


@pytest.mark.parametrize("n,per,st", [((5, 6), (False, True), 3), ((5, 5), (False, False), 5),
                                      ((4, 4, 5), (False, True, False), 3)])
def test_gradients_match_dense_autograd(n, per, st):
    """The OptNet formulas after Eq. 11 against reverse-mode autograd through a
    dense FP64 normal-equation solve on a tiny grid."""
    w = wl.random_problem(5, n, per, st)
    N = w.npoints
    V = asm.n_vars(len(n))
    c = w.full_coeff()[:, 0]
    A, d, kind, owner = asm.assemble(w.geom, c, w.rhs[0], w.omega[0])
    z, lam, kkt = osv.solve_lsq(A, d)
    L, g = _loss_and_g(z, w.target[0], N)
    dz, dlam = og.adjoint(kkt, g)
    dc, db, dom = og.gradients(w.geom, A, d, kind, owner, z, lam, dz, dlam)

    eq = np.flatnonzero(kind == asm.E)
    bcr = np.flatnonzero(kind == asm.BC)
    base = torch.tensor(A.toarray())
    ct = torch.tensor(c, requires_grad=True)
    bt = torch.tensor(w.rhs[0], requires_grad=True)
    ot = torch.tensor(w.omega[0], requires_grad=True)
    pe = torch.tensor(owner[eq])
    mask = torch.zeros_like(base)
    mask[eq] = 1.0
    Aeq = torch.zeros_like(base)
    for v in range(V):
        Aeq = Aeq.index_put((torch.tensor(eq), v * N + pe), ct[v][pe])
    At = base * (1 - mask) + Aeq
    dt = torch.zeros(A.shape[0], dtype=torch.float64)
    dt = dt.index_put((torch.tensor(eq),), bt[pe])
    dt = dt.index_put((torch.tensor(bcr),), ot[torch.tensor(owner[bcr])])
    zt = torch.linalg.solve(At.T @ At, At.T @ dt)
    Lt = ((zt[:N] - torch.tensor(w.target[0])) ** 2).mean()
    Lt.backward()
    assert abs(Lt.item() - L) < 1e-10 * max(1, abs(L))
    for mine, ref in ((dc, ct.grad), (db, bt.grad), (dom, ot.grad)):
        ref = ref.numpy()
        assert np.linalg.norm(mine - ref) <= 1e-7 * max(1e-30, np.linalg.norm(ref))


def test_gradients_match_finite_differences():
    """Central differences of L through the oracle's solve at random coordinates."""
    w = wl.random_problem(9, (6, 8), (False, True), 3)
    N = w.npoints
    c = w.full_coeff()[:, 0]

    def loss(c_, b_, o_):
        A, d, *_ = asm.assemble(w.geom, c_, b_, o_)
        z, _, _ = osv.solve_lsq(A, d)
        return _loss_and_g(z, w.target[0], N)[0]

    A, d, kind, owner = asm.assemble(w.geom, c, w.rhs[0], w.omega[0])
    z, lam, kkt = osv.solve_lsq(A, d)
    _, g = _loss_and_g(z, w.target[0], N)
    dz, dlam = og.adjoint(kkt, g)
    dc, db, dom = og.gradients(w.geom, A, d, kind, owner, z, lam, dz, dlam)
    rng = np.random.default_rng(0)
    bnd = np.flatnonzero(asm.boundary_mask(w.geom))
    h = 1e-4
    tol = lambda fd, ref: 1e-5 * max(abs(fd), 1e-2 * np.abs(ref).max())
    for _ in range(8):
        v, p = rng.integers(0, 5), rng.integers(0, N)
        cp, cm = c.copy(), c.copy()
        cp[v, p] += h; cm[v, p] -= h
        fd = (loss(cp, w.rhs[0], w.omega[0]) - loss(cm, w.rhs[0], w.omega[0])) / (2 * h)
        assert abs(fd - dc[v, p]) <= tol(fd, dc)
        p = rng.integers(0, N)
        bp, bm = w.rhs[0].copy(), w.rhs[0].copy()
        bp[p] += h; bm[p] -= h
        fd = (loss(c, bp, w.omega[0]) - loss(c, bm, w.omega[0])) / (2 * h)
        assert abs(fd - db[p]) <= tol(fd, db)
        p = bnd[rng.integers(0, len(bnd))]
        op, om = w.omega[0].copy(), w.omega[0].copy()
        op[p] += h; om[p] -= h
        fd = (loss(c, w.rhs[0], op) - loss(c, w.rhs[0], om)) / (2 * h)
        assert abs(fd - dom[p]) <= tol(fd, dom)


def test_gradient_identities():
    """d_lambda = -A d_z (Eq. 11, first block row) and dl/dd = A d_z."""
    w = wl.random_problem(2, (5, 6, 6), (False, True, True), 3)
    N = w.npoints
    A, d, kind, owner = asm.assemble(w.geom, w.full_coeff()[:, 0], w.rhs[0], w.omega[0])
    z, lam, kkt = osv.solve_lsq(A, d)
    _, g = _loss_and_g(z, w.target[0], N)
    dz, dlam = og.adjoint(kkt, g)
    assert np.linalg.norm(dlam + A @ dz) <= 1e-9 * np.linalg.norm(dlam)
    assert np.linalg.norm(A.T @ (A @ dz) - g) <= 1e-9 * np.linalg.norm(g)


@pytest.mark.parametrize("n,per,st", [((6, 6), (False, False), 3), ((6, 8), (False, True), 5),
                                      ((4, 5, 6), (False, True, False), 3),
                                      ((5, 6, 6), (False, True, True), 5)])
def test_elimination_route_matches_dense_lstsq(n, per, st):
    """The block-elimination solve of Eq. 9 against numpy's dense least
    squares, for the forward problem and for an adjoint right-hand side."""
    w = wl.random_problem(13, n, per, st, final_time_rows=True)
    V = asm.n_vars(len(n))
    A, d, kind, owner = asm.assemble(w.geom, w.full_coeff()[:, 0], w.rhs[0], w.omega[0])
    z, lam, el = osv.solve_lsq_elim(A, d, V)
    Ad = A.toarray()
    zref = np.linalg.lstsq(Ad, d, rcond=None)[0]
    assert np.linalg.norm(z - zref) <= 1e-10 * np.linalg.norm(zref)
    g = np.random.default_rng(1).normal(size=A.shape[1])
    dz, dlam = og.adjoint_elim(el, g)
    dzref = np.linalg.solve(Ad.T @ Ad, g)
    assert np.linalg.norm(dz - dzref) <= 1e-9 * np.linalg.norm(dzref)
    assert np.linalg.norm(dlam + Ad @ dzref) <= 1e-9 * np.linalg.norm(Ad @ dzref)


def test_elimination_route_matches_kkt_route_3d():
    w = wl.reaction_diffusion_2d(batch=1, n=(8, 8, 8))
    A, d, kind, owner = asm.assemble(w.geom, w.full_coeff()[:, 0], w.rhs[0], w.omega[0])
    z1, lam1, _ = osv.solve_lsq(A, d)
    z2, lam2, _ = osv.solve_lsq_elim(A, d, 7)
    assert np.linalg.norm(z1 - z2) <= 1e-9 * np.linalg.norm(z1)
    assert osv.normal_residual(A, d, z2) < 1e-12


# ------------------------------------------- data with a known LS solution
@pytest.mark.parametrize("n,per,final", [((6, 7), (False, False), False), ((6, 8), (False, True), True),
                                         ((5, 6, 8), (False, True, False), False),
                                         ((5, 6, 8), (False, False, False), True),
                                         ((5, 8, 8), (False, True, True), False),
                                         ((4, 3, 5), (False, False, True), False)])
def test_manufactured_data_is_consistent_for_any_u(n, per, final):
    """oracle.manufactured: for a white-noise u (no smoothness at all) and
    random coefficient fields, the assembled system (Eqs. 3-8) with the
    manufactured b and omega has zero residual at z_e, and the saddle-point
    solve (Eq. 10) returns z_e with a zero dual.  A wrong weight, sign or
    step power in any difference form, or a missing edge case, leaves a
    residual of order one."""
    w = wl.random_problem(51, n, per, final_time_rows=final)
    rng = np.random.default_rng(52)
    N = int(np.prod(n))
    c = w.full_coeff()[:, 0]
    u = rng.normal(size=N)
    from oracle import manufactured as mf
    z, b, om = mf.consistent_data(w.geom, c, u)
    assert np.array_equal(z[0], u)
    A, d, kind, owner = asm.assemble(w.geom, c, b, om)
    assert np.linalg.norm(A @ z.ravel() - d) <= 1e-13 * np.linalg.norm(d)
    zs, lam, kkt = osv.solve_lsq(A, d)
    assert np.linalg.norm(zs - z.ravel()) <= 1e-10 * np.linalg.norm(z)
    assert np.abs(lam).max() <= 1e-9 * np.abs(d).max()
    # the backward system (Eq. 11) with g = A^T A z' returns z' for any z'
    zp = rng.normal(size=A.shape[1])
    dz, dlam = og.adjoint(kkt, A.T @ (A @ zp))
    assert np.linalg.norm(dz - zp) <= 1e-9 * np.linalg.norm(zp)
    assert np.linalg.norm(dlam + A @ zp) <= 1e-9 * np.linalg.norm(A @ zp)


def test_manufactured_data_matches_polynomial_derivatives():
    """On a separable quadratic in every non-periodic dimension the difference
    forms are exact, so the manufactured derivative unknowns equal the
    analytic derivatives (pins the 1/s, 1/s^2 scaling and the variable order)."""
    from oracle import manufactured as mf
    g = _geom((5, 6, 7), (False, False, False), lengths=(1.0, 2.0, 0.5))
    t, x, y = (np.arange(k) * s for k, s in zip(g["n"], g["step"]))
    T, X, Y = np.meshgrid(t, x, y, indexing="ij")
    u = (1 + 2 * T - 3 * T * T) * (0.5 - X + 0.25 * X * X) * (2 + Y + 4 * Y * Y)
    z = mf.consistent_z(g, u.ravel())
    pt, px, py = (1 + 2 * T - 3 * T * T), (0.5 - X + 0.25 * X * X), (2 + Y + 4 * Y * Y)
    ref = [u, (2 - 6 * T) * px * py, -6 * px * py, pt * (-1 + 0.5 * X) * py, pt * 0.5 * py,
           pt * px * (1 + 8 * Y), pt * px * 8]
    for v in range(7):
        np.testing.assert_allclose(z[v], ref[v].ravel(), rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("n,per,final", [((6, 8), (False, True), False), ((5, 6, 8), (False, True, True), False),
                                         ((5, 6, 7), (False, False, False), True)])
def test_eliminated_pair_solves_the_adjoint_system(n, per, final):
    """oracle.manufactured.eliminated_pair: g vanishes on every derivative
    unknown, and the backward saddle-point system (Eq. 11) with this g returns
    z_e (the oracle's KKT route, which never forms the point blocks)."""
    from oracle import manufactured as mf
    w = wl.random_problem(61, n, per, final_time_rows=final)
    c = w.full_coeff()[:, 0]
    A, d, kind, owner = asm.assemble(w.geom, c, w.rhs[0], w.omega[0])
    V, N = asm.n_vars(len(n)), int(np.prod(n))
    u = wl.low_mode_field(np.random.default_rng(62), w.geom)
    z, g, resid = mf.eliminated_pair(A, V, u)
    assert resid < 1e-12
    assert np.array_equal(z[:N], u) and not np.any(g[N:])
    kkt = osv.KKT(A)
    dz, dlam = og.adjoint(kkt, g)
    assert np.linalg.norm(dz - z) <= 1e-9 * np.linalg.norm(z)
