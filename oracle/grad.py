"""Adjoint solve and parameter gradients (Section 3, Eq. 11 and the formulas
after it), in FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Given g_z = dl/dz*, the backward saddle-point system (Eq. 11)
    [ I   A ] [d_lambda]   [  0  ]
    [ A^T 0 ] [  d_z   ] = [ -g_z]
gives A^T A d_z = g_z and d_lambda = -A d_z.  Following OptNet, the gradients
with respect to the data of the least-squares problem are
    dl/dA = d_lambda z*^T + lambda* d_z^T,        dl/dd = -d_lambda.
The PDE data enter A and d only through the equation rows (Eq. 3: entry
c_{v,i} at column (v, i), right-hand side b_i) and the boundary rows (Eq. 4:
right-hand side omega_i), so
    dl/dc_{v,i} = d_lambda_{E,i} z*_{v,i} + lambda*_{E,i} d_z_{v,i}
    dl/db_i     = -d_lambda_{E,i}
    dl/domega_i = -d_lambda_{BC,i}            (i in the boundary set)
"""
from __future__ import annotations

import numpy as np

from . import assemble as asm
from .solve import KKT


def adjoint(kkt: KKT, g_z):
    """Eq. 11: returns (d_z, d_lambda)."""
    dlam, dz = kkt.solve(np.zeros(kkt.nc), -np.asarray(g_z, dtype=np.float64))
    return dz, dlam


def gradients(geom, A, d, kind, owner, z, lam, dz, dlam):
    """Per-point gradients from the formulas after Eq. 11.

    Returns (dcoeff (V, N), db (N,), domega (N,)); domega is zero off the
    boundary set."""
    n = tuple(geom["n"])
    N = int(np.prod(n))
    V = asm.n_vars(len(n))
    zv = np.asarray(z).reshape(V, N)
    dzv = np.asarray(dz).reshape(V, N)
    eq = np.flatnonzero(kind == asm.E)
    pe = owner[eq]
    dcoeff = np.zeros((V, N))
    dcoeff[:, pe] = dlam[eq][None, :] * zv[:, pe] + lam[eq][None, :] * dzv[:, pe]
    db = np.zeros(N)
    db[pe] = -dlam[eq]
    bc = np.flatnonzero(kind == asm.BC)
    domega = np.zeros(N)
    domega[owner[bc]] = -dlam[bc]
    return dcoeff, db, domega


def dense_dA(A, z, lam, dz, dlam):
    """dl/dA as a dense matrix (tiny grids only): d_lambda z^T + lambda d_z^T."""
    return np.outer(dlam, z) + np.outer(lam, dz)


def adjoint_elim(elim, g_z):
    """Eq. 11 through NormalElim: A^T A d_z = g_z, d_lambda = -A d_z."""
    dz = elim.solve(np.asarray(g_z, dtype=np.float64))
    return dz, -(elim.A @ dz)
