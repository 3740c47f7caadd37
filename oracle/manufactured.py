"""Data whose least-squares solution is known exactly, at any grid size
(Section 3, Eqs. 3-9), in FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

With three-point derivative rows, the rows of Eqs. 5-7 along one dimension
never contradict each other, whatever the values of u, once the derivative
unknowns take the values of the difference forms of Eq. 5:
  * interior / periodic point: the forward and backward Taylor rows (Eqs. 6-7)
    u_i +- s u'_i + s^2/2 u''_i = u_{i+-1} are solved by
    s u'_i = (u_{i+1} - u_{i-1}) / 2 and s^2 u''_i = u_{i+1} - 2 u_i + u_{i-1}
    (their half sum and half difference), which are the central forms of the
    two derivative rows;
  * first point of a non-periodic dimension (no backward row): the forward
    Taylor row and the one-sided second-difference row
    s^2 u''_0 = u_0 - 2 u_1 + u_2 give s u'_0 = (-3 u_0 + 4 u_1 - u_2) / 2,
    the one-sided first-difference row; mirrored at the last point.
So for ANY u, the vector z_e = (u, u-derivatives := difference forms / s^k)
satisfies every derivative and Taylor row exactly.  Taking the equation rows'
right-hand side b := sum_v c_v z_e,v (Eq. 3) and the Dirichlet values
omega := u (Eq. 4) makes A z_e = d a consistent system, so z_e is its
least-squares solution (Eq. 9, A of full column rank).  For the backward
system of Eq. 11, any z and g := A^T A z give d_z = z.

This is the plain definition written out per dimension with numpy; it shares
nothing with the CUDA path.  Five-point rows (stencil 5) are not covered:
their interior forms are not combinations of the Taylor rows.
"""
from __future__ import annotations

import numpy as np

from . import assemble as asm


def _diff_forms(u, axis, periodic):
    """(s u', s^2 u'') along `axis` of the grid array u: three-point central
    forms, wrapped when periodic, second-order one-sided forms at the two
    edges of a non-periodic axis (Eq. 5 and the edge reading above)."""
    if periodic:
        up = np.roll(u, -1, axis)
        um = np.roll(u, 1, axis)
        return 0.5 * (up - um), up - 2.0 * u + um
    n = u.shape[axis]
    a1 = np.empty_like(u)
    a2 = np.empty_like(u)
    sl = lambda i: tuple(slice(None) if k != axis else i for k in range(u.ndim))
    mid = sl(slice(1, n - 1))
    a1[mid] = 0.5 * (u[sl(slice(2, n))] - u[sl(slice(0, n - 2))])
    a2[mid] = u[sl(slice(2, n))] - 2.0 * u[mid] + u[sl(slice(0, n - 2))]
    u0, u1, u2 = u[sl(0)], u[sl(1)], u[sl(2)]
    a1[sl(0)] = -1.5 * u0 + 2.0 * u1 - 0.5 * u2
    a2[sl(0)] = u0 - 2.0 * u1 + u2
    v0, v1, v2 = u[sl(n - 1)], u[sl(n - 2)], u[sl(n - 3)]
    a1[sl(n - 1)] = 1.5 * v0 - 2.0 * v1 + 0.5 * v2
    a2[sl(n - 1)] = v0 - 2.0 * v1 + v2
    return a1, a2


def consistent_z(geom, u):
    """z_e (V, N) for the grid values u (N,): u and, per dimension d (time
    first), its first and second derivative taken as the difference forms
    divided by s_d and s_d^2."""
    n = tuple(geom["n"])
    assert geom.get("stencil", 3) == 3, "three-point derivative rows only"
    D = len(n)
    ug = np.asarray(u, dtype=np.float64).reshape(n)
    z = np.empty((asm.n_vars(D), ug.size))
    z[0] = ug.ravel()
    for d in range(D):
        s = geom["step"][d]
        a1, a2 = _diff_forms(ug, d, geom["periodic"][d])
        z[asm.first(d)] = a1.ravel() / s
        z[asm.second(d)] = a2.ravel() / (s * s)
    return z


def consistent_data(geom, coeff, u):
    """(z_e, b, omega) with A z_e = d exactly: b_i = sum_v c_{v,i} z_e,{v,i}
    (Eq. 3) and omega = u (Eq. 4; only boundary points are read).
    coeff: (V, N) per-point coefficients."""
    z = consistent_z(geom, u)
    b = np.einsum("vn,vn->n", np.asarray(coeff, dtype=np.float64), z)
    return z, b, z[0].copy()


def _point_blocks(A, nvar):
    """(A_u, A_w, blocks): the u columns and the derivative columns of A, and
    the (V-1) x (V-1) block of M_ww = A_w^T A_w of every point.  The
    derivative unknowns of a point appear only in that point's rows (Eqs. 3
    and 5-7), so M_ww is block diagonal; only products with A and A^T and
    these blocks are formed (never the whole M = A^T A), which keeps this
    within reach at the full benchmark sizes."""
    import scipy.sparse as sp
    A = sp.csr_matrix(A)
    N = A.shape[1] // nvar
    nb = nvar - 1
    Au = A[:, :N]
    Aw = A[:, N:]
    Mww = (Aw.T @ Aw).tocoo()
    pi, vi = Mww.row % N, Mww.row // N
    pj, vj = Mww.col % N, Mww.col // N
    assert np.all(pi == pj), "derivative unknowns must be point-local"
    blk = np.zeros((N, nb, nb))
    np.add.at(blk, (pi, vi, vj), Mww.data)
    return A, Au, Aw, blk


def eliminate_w(A, nvar, u, blocks=None):
    """Derivative unknowns w = -M_ww^{-1} M_wu u for the u values u (N,):
    the minimiser of ||A (u, w)||^2 over w, point by point (M = A^T A).  For
    any adjoint source g that vanishes on the derivative unknowns, the
    solution d_z of A^T A d_z = g (Eq. 11) has exactly these derivative
    unknowns for its own u part.  Returned as (V-1, N); the block solves are
    refined once in FP64."""
    A, Au, Aw, blk = blocks if blocks is not None else _point_blocks(A, nvar)
    N, nb = blk.shape[0], blk.shape[1]
    u = np.asarray(u, dtype=np.float64)
    rhs = -(Aw.T @ (Au @ u)).reshape(nb, N).T            # -M_wu u, one row per point
    w = np.linalg.solve(blk, rhs[..., None])[..., 0]
    w += np.linalg.solve(blk, (rhs - np.einsum("pij,pj->pi", blk, w))[..., None])[..., 0]
    return w.T


def eliminated_pair(A, nvar, u):
    """(z_e, g, resid) with A^T A z_e = g exactly and g zero on every
    derivative unknown, for the grid values u (N,) of the u unknowns (Eq. 11
    with an adjoint source on u only, the form a loss on u produces):
    z_e = (u, eliminate_w(u)), g = A^T A z_e.  The w part of g that rounding
    leaves is returned as `resid` (relative to the terms it balances) and
    g_w is then set to zero exactly."""
    blocks = _point_blocks(A, nvar)
    A, Au, Aw, blk = blocks
    N = blk.shape[0]
    u = np.asarray(u, dtype=np.float64)
    z = np.concatenate([u, eliminate_w(A, nvar, u, blocks).ravel()])
    g = A.T @ (A @ z)
    scale = np.linalg.norm(Aw.T @ (Au @ u))
    resid = float(np.linalg.norm(g[N:]) / (scale if scale > 0 else 1.0))
    g[N:] = 0.0
    return z, g, resid
