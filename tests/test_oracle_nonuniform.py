"""Pins of the oracle's per-interval-step assembly (oracle/nonuniform.py):
unequal steps, Neumann and mixed boundary rows, and dl/dh.

Each checks it against something other than itself: the uniform assembly
(pinned on its own in test_oracle.py) for equal steps, exactness on
quadratics (which fixes every three-point weight on any grid), convergence to
an analytic heat mode on a stretched grid with Neumann and with mixed
boundary data, and central finite differences of the loss through the
oracle's solve for the step gradients.
"""
import math

import numpy as np
import pytest

from oracle import assemble as asm
from oracle import grad as og
from oracle import nonuniform as nu
from oracle import solve as osv
from paper_2502_18377_b300 import workloads as wl


def _random_intervals(rng, geom, spread=0.4):
    """Per-dimension steps around the uniform one, each within +-spread."""
    return [h * rng.uniform(1 - spread, 1 + spread, size=h.size) for h in nu.uniform_intervals(geom)]


def _face_dims(geom):
    """For every point: the dimension of its boundary row (-1 if none), with
    the faces taken in the order t = 0, t = t_f (when present), then the
    spatial dimensions lower face first; the first face a point is on wins."""
    n = geom["n"]
    idx = asm.multi_index(n)
    out = np.full(idx.shape[0], -1)
    faces = [(0, 0)]
    if geom.get("final_time_rows", False):
        faces.append((0, n[0] - 1))
    for d in range(1, len(n)):
        if not geom["periodic"][d]:
            faces += [(d, 0), (d, n[d] - 1)]
    for d, k in faces:
        sel = (idx[:, d] == k) & (out < 0)
        out[sel] = d
    return out


def _exact_quadratic(rng, geom, intervals):
    """z of a separable u = prod_d q_d(x_d), q_d a random quadratic in the
    coordinate x_d = cumulative sum of the steps (a constant along periodic
    dimensions, where no quadratic is periodic)."""
    n = geom["n"]
    D = len(n)
    fac = []
    for d in range(D):
        x = np.concatenate([[0.0], np.cumsum(intervals[d])])[: n[d]]
        if geom["periodic"][d]:
            c = rng.uniform(0.5, 1.5)
            fac.append((np.full(n[d], c), np.zeros(n[d]), np.zeros(n[d])))
        else:
            a, b, c = rng.uniform(-1, 1, size=3)
            fac.append((a + b * x + c * x * x, b + 2 * c * x, np.full(n[d], 2 * c)))

    def outer(parts):
        out = parts[0]
        for p in parts[1:]:
            out = np.multiply.outer(out, p)
        return out.ravel()

    V = asm.n_vars(D)
    z = np.empty((V, int(np.prod(n))))
    z[0] = outer([f[0] for f in fac])
    for d in range(D):
        for k, var in ((1, asm.first(d)), (2, asm.second(d))):
            z[var] = outer([fac[e][k] if e == d else fac[e][0] for e in range(D)])
    return z


def _boundary_data(geom, z):
    """omega = alpha u + beta du/dx_d at each boundary point, d the dimension
    of its row and (alpha, beta) that dimension's boundary kind."""
    dims = _face_dims(geom)
    bc = geom.get("bc", {})
    om = np.zeros(z.shape[1])
    for p in np.flatnonzero(dims >= 0):
        d = dims[p]
        a, b = bc.get(d, (1.0, 0.0)) if d > 0 else (1.0, 0.0)
        om[p] = a * z[0, p] + (b * z[asm.first(d), p] if d > 0 else 0.0)
    return om


def _loss_and_g(z, tgt, N):
    r = z[:N] - tgt
    g = np.zeros_like(z)
    g[:N] = 2 * r / N
    return float((r * r).mean()), g


# ---------------------------------------------------- equal steps = uniform
@pytest.mark.parametrize("n,per,final", [((6, 7), (False, False), False), ((6, 8), (False, True), True),
                                         ((5, 6, 8), (False, True, False), False),
                                         ((5, 6, 7), (False, False, False), True),
                                         ((4, 5, 6), (False, True, True), False)])
def test_equal_steps_reproduce_the_uniform_assembly(n, per, final):
    """With every interval equal to the uniform step, the system is the
    uniform one up to the order of its rows: same shape and nonzero count,
    same rows per family, same normal matrix A^T A and same A^T d."""
    w = wl.random_problem(3, n, per, final_time_rows=final)
    c = w.full_coeff()[:, 0]
    A1, d1, k1, o1 = asm.assemble(w.geom, c, w.rhs[0], w.omega[0])
    A2, d2, k2, o2 = nu.assemble(w.geom, c, w.rhs[0], w.omega[0])
    assert A1.shape == A2.shape and A1.nnz == A2.nnz
    assert np.bincount(k1).tolist() == np.bincount(k2).tolist()
    for fam in np.unique(k1):
        assert sorted(o1[k1 == fam].tolist()) == sorted(o2[k2 == fam].tolist())
    M1, M2 = (A1.T @ A1).toarray(), (A2.T @ A2).toarray()
    assert np.abs(M1 - M2).max() <= 1e-13 * np.abs(M1).max()
    assert np.abs(A1.T @ d1 - A2.T @ d2).max() <= 1e-13 * max(1.0, np.abs(A1.T @ d1).max())


def test_five_point_stencil_is_refused():
    w = wl.random_problem(3, (6, 8), (False, True), stencil=5)
    with pytest.raises(ValueError):
        nu.assemble(w.geom, w.full_coeff()[:, 0], w.rhs[0], w.omega[0])


# ------------------------------------------------- exactness on quadratics
@pytest.mark.parametrize("n,per,bc", [
    ((6, 7), (False, False), {}),
    ((6, 7), (False, False), {1: (0.0, 1.0)}),
    ((7, 6), (False, False), {1: (0.7, -0.4)}),
    ((6, 8), (False, True), {}),
    ((5, 6, 7), (False, False, False), {1: (0.0, 1.0), 2: (1.0, 0.5)}),
    ((5, 6, 7), (False, True, False), {2: (0.0, 1.0)}),
])
def test_quadratics_are_exact_on_unequal_steps(n, per, bc):
    """The three-point forms on unequal steps (central inside, one-sided at
    the edges) and the Taylor rows are exact for quadratics, and Neumann and
    mixed rows are exact by construction: a separable quadratic u with its
    derivatives, b = sum_v c_v z_v and the boundary data of its own values has
    zero residual, so the least-squares solution is that z.  A wrong weight,
    sign, step or neighbour in any family leaves a residual here."""
    rng = np.random.default_rng(11)
    geom = dict(wl.random_problem(0, n, per).geom, bc=bc)
    iv = _random_intervals(rng, geom)
    z = _exact_quadratic(rng, geom, iv)
    V, N = z.shape
    c = rng.uniform(-1, 1, size=(V, N))
    c[1] = rng.uniform(0.5, 1.5, size=N)
    b = (c * z).sum(0)
    om = _boundary_data(geom, z)
    A, d, kind, owner = nu.assemble(geom, c, b, om, iv)
    r = A @ z.ravel() - d
    assert np.abs(r).max() < 1e-10 * max(1.0, np.abs(z).max())
    zs, lam, _ = osv.solve_lsq(A, d)
    assert np.linalg.norm(zs - z.ravel()) <= 1e-8 * np.linalg.norm(z)


def test_boundary_rows_follow_the_face_order():
    """One boundary row per boundary point; its kind and target variable
    follow the face order t = 0, t = t_f, spatial dimensions lower face first."""
    geom = dict(wl.random_problem(0, (5, 6, 7), (False, False, False), final_time_rows=True).geom,
                bc={1: (0.0, 1.0), 2: (0.3, 0.8)})
    N = 5 * 6 * 7
    A, d, kind, owner = nu.assemble(geom, np.ones((7, N)), np.zeros(N), np.arange(N, dtype=float))
    dims = _face_dims(geom)
    bc = np.flatnonzero(kind == asm.BC)
    assert sorted(owner[bc].tolist()) == np.flatnonzero(dims >= 0).tolist()
    for r in bc:
        p = owner[r]
        row = A.getrow(r)
        cols = dict(zip(row.indices.tolist(), row.data.tolist()))
        dd = dims[p]
        a, b = geom["bc"].get(dd, (1.0, 0.0)) if dd > 0 else (1.0, 0.0)
        want = {}
        if a:
            want[p] = a
        if b:
            want[asm.first(dd) * N + p] = b
        assert cols == pytest.approx(want)
        assert d[r] == p


# ------------------------------------------- convergence on a stretched grid
def _stretched(m, eps=0.1):
    """Intervals of x_j = s_j + eps sin(2 pi s_j), s_j = j / (m - 1): a smooth,
    monotone stretching of [0, 1] with steps varying by a factor ~1.9."""
    s = np.arange(m) / (m - 1)
    x = s + eps * np.sin(2 * math.pi * s)
    return x, np.diff(x)


@pytest.mark.parametrize("bc", [(0.0, 1.0), (1.0, 0.6)])
def test_heat_mode_converges_on_a_stretched_grid(bc):
    """u = exp(-nu k^2 t) cos(k x + phi) solves u_t - nu u_xx = 0.  On a
    stretched x grid, with Neumann (phi = 0, so u_x = 0 at both ends: zero
    data) or mixed boundary data alpha u + beta u_x from u, the least-squares
    u approaches it as the grid refines, at second order."""
    nuv, k = 0.05, math.pi
    phi = 0.0 if bc == (0.0, 1.0) else 0.4
    errs = []
    for m in (12, 24, 48):
        geom = dict(n=(m, m), step=(1.0 / (m - 1), 1.0 / (m - 1)), periodic=(False, False), stencil=3,
                    final_time_rows=False, bc={1: bc})
        x, hx = _stretched(m)
        t = np.arange(m) / (m - 1)
        ht = np.diff(t)
        T, X = np.meshgrid(t, x, indexing="ij")
        decay = np.exp(-nuv * k * k * T)
        u = decay * np.cos(k * X + phi)
        ux = -k * decay * np.sin(k * X + phi)
        N = m * m
        z = np.zeros((5, N))
        z[0], z[3] = u.ravel(), ux.ravel()
        om = _boundary_data(geom, z)
        c = np.zeros((5, N)); c[1] = 1.0; c[4] = -nuv
        A, d, kind, owner = nu.assemble(geom, c, np.zeros(N), om, [ht, hx])
        zs, _, _ = osv.solve_lsq(A, d)
        errs.append(np.linalg.norm(zs[:N] - u.ravel()) / np.linalg.norm(u))
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[2] < 5e-3, errs
    assert math.log2(errs[1] / errs[2]) > 1.5, errs


# --------------------------------------------------------- step gradients
@pytest.mark.parametrize("n,per,bc,final", [
    ((6, 8), (False, True), {}, False),
    ((6, 7), (False, False), {1: (0.0, 1.0)}, True),
    ((4, 5, 6), (False, False, True), {1: (0.8, 0.5)}, False),
])
def test_step_gradients_match_finite_differences(n, per, bc, final):
    """dl/dh from the gradient formula after Eq. 11 against central
    differences of the loss through the oracle's solve, for every interval
    of every dimension (time included)."""
    rng = np.random.default_rng(5)
    w = wl.random_problem(9, n, per, final_time_rows=final)
    geom = dict(w.geom, bc=bc)
    N = w.npoints
    c, b, om, tgt = w.full_coeff()[:, 0], w.rhs[0], w.omega[0], w.target[0]
    iv = _random_intervals(rng, geom, spread=0.3)

    def loss(iv_):
        A, d, *_ = nu.assemble(geom, c, b, om, iv_)
        z, _, _ = osv.solve_lsq(A, d)
        return _loss_and_g(z, tgt, N)[0]

    A, d, kind, owner = nu.assemble(geom, c, b, om, iv)
    z, lam, kkt = osv.solve_lsq(A, d)
    _, g = _loss_and_g(z, tgt, N)
    dz, dlam = og.adjoint(kkt, g)
    dh = nu.step_gradients(geom, c, b, om, iv, z, lam, dz, dlam)
    assert [x.shape for x in dh] == [h.shape for h in iv]
    for dim, h in enumerate(iv):
        scale = np.abs(dh[dim]).max()
        assert scale > 0
        for k in range(h.size):
            eps = 1e-4 * h[k]
            ip = [x.copy() for x in iv]
            im = [x.copy() for x in iv]
            ip[dim][k] += eps
            im[dim][k] -= eps
            fd = (loss(ip) - loss(im)) / (2 * eps)
            assert abs(fd - dh[dim][k]) <= 2e-6 * scale, (dim, k, fd, dh[dim][k])
