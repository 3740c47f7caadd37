"""Exact FP64 least-squares solve of A z = d (Section 3, Eqs. 8-10).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The forward solution is z* = argmin ||A z - d||_2, the solution of the normal
equations A^T A z = A^T d (Eq. 9).  It is computed from the saddle-point form
of Eq. 10,
    [ I   A ] [lambda*]   [d]
    [ A^T 0 ] [  z*   ] = [0],
with a sparse LU factorisation (SuperLU), which avoids squaring the condition
number of A.  The dual is lambda* = d - A z* (first block row of Eq. 10).
`solve_normal` factorises A^T A directly and serves as a cross-check.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


class KKT:
    """LU factorisation of the saddle-point matrix of Eqs. 10-11 for one A."""

    def __init__(self, A):
        A = sp.csr_matrix(A)
        nc, nv = A.shape
        self.A = A
        self.nc, self.nv = nc, nv
        K = sp.bmat([[sp.identity(nc, format="csr"), A], [A.T, None]], format="csc")
        self.lu = spla.splu(K, permc_spec="COLAMD")

    def solve(self, top, bottom):
        """Solve [I A; A^T 0] [x; y] = [top; bottom]; returns (x, y)."""
        rhs = np.concatenate([np.asarray(top, dtype=np.float64),
                              np.asarray(bottom, dtype=np.float64)])
        sol = self.lu.solve(rhs)
        return sol[: self.nc], sol[self.nc:]


def solve_lsq(A, d, kkt=None):
    """Forward pass (Eq. 10): returns (z*, lambda*, kkt factorisation)."""
    kkt = kkt or KKT(A)
    lam, z = kkt.solve(d, np.zeros(kkt.nv))
    return z, lam, kkt


def solve_normal(A, d):
    """Eq. 9 solved by sparse LU of A^T A (cross-check of solve_lsq)."""
    A = sp.csr_matrix(A)
    M = (A.T @ A).tocsc()
    return spla.splu(M, permc_spec="COLAMD").solve(A.T @ d)


def normal_residual(A, d, z):
    """Relative normal-equation residual ||A^T (d - A z)|| / ||A^T d||."""
    A = sp.csr_matrix(A)
    r = A.T @ (d - A @ z)
    den = np.linalg.norm(A.T @ d)
    return float(np.linalg.norm(r) / (den if den > 0 else 1.0))
