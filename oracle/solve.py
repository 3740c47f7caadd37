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


class NormalElim:
    """Eq. 9 solved by block Gaussian elimination, for grids where the
    saddle-point LU fills in too much.

    The derivative unknowns of a grid point appear only in rows owned by that
    point (Eqs. 3 and 5-7 at that point), so in M = A^T A they form a block
    diagonal of (V-1) x (V-1) blocks.  Eliminating them leaves the Schur
    complement S = M_uu - M_uw M_ww^{-1} M_wu on the u unknowns, which is
    factorised by sparse LU; the derivative unknowns follow by back
    substitution.  Two steps of FP64 iterative refinement against the
    assembled A remove the rounding that forming A^T A introduces.
    """

    def __init__(self, A, nvar):
        A = sp.csr_matrix(A)
        self.A = A
        self.At = A.T.tocsr()
        nv = A.shape[1]
        N = nv // nvar
        self.N, self.V = N, nvar
        M = (self.At @ A).tocsr()
        u = np.arange(N)
        w = np.arange(N, nv)
        Muu = M[u][:, u]
        Muw = M[u][:, w]
        Mww = M[w][:, w].tocoo()
        # block-diagonal inverse of M_ww: blocks indexed by grid point
        nb = nvar - 1
        blk = np.zeros((N, nb, nb))
        bi, bj = Mww.row, Mww.col
        pi, vi = bi % N, bi // N
        pj, vj = bj % N, bj // N
        assert np.all(pi == pj), "derivative unknowns must be point-local"
        np.add.at(blk, (pi, vi, vj), Mww.data)
        inv = np.linalg.inv(blk)
        rows = (np.arange(nb)[None, :, None] * N + np.arange(N)[:, None, None])
        cols = (np.arange(nb)[None, None, :] * N + np.arange(N)[:, None, None])
        rows, cols = np.broadcast_arrays(rows, cols)
        self.Mww_inv = sp.csr_matrix((inv.ravel(), (rows.ravel(), cols.ravel())),
                                     shape=(nb * N, nb * N))
        self.Muw = Muw
        self.Mwu = Muw.T.tocsr()
        S = (Muu - Muw @ self.Mww_inv @ self.Mwu).tocsc()
        self.S = S
        self.lu = spla.splu(S, permc_spec="COLAMD")

    def reduced_rhs(self, rhs):
        """u-part of the eliminated right-hand side: rhs_u - M_uw M_ww^{-1} rhs_w."""
        N = self.N
        return rhs[:N] - self.Muw @ (self.Mww_inv @ rhs[N:])

    def solve_normal(self, rhs):
        """One elimination solve of A^T A z = rhs."""
        N = self.N
        ru, rw = rhs[:N], rhs[N:]
        u = self.lu.solve(ru - self.Muw @ (self.Mww_inv @ rw))
        w = self.Mww_inv @ (rw - self.Mwu @ u)
        return np.concatenate([u, w])

    def solve(self, rhs, refine=2):
        """A^T A z = rhs with FP64 iterative refinement."""
        z = self.solve_normal(rhs)
        for _ in range(refine):
            z = z + self.solve_normal(rhs - self.At @ (self.A @ z))
        return z


def solve_lsq_elim(A, d, nvar, elim=None):
    """Forward pass via NormalElim: returns (z*, lambda* = d - A z*, elim)."""
    elim = elim or NormalElim(A, nvar)
    z = elim.solve(elim.At @ d)
    return z, d - elim.A @ z, elim
