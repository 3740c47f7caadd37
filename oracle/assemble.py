"""Assembly of the constraint system A z = d of Section 3 (Eqs. 3-8), in FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Unknowns (Section 3, "Variables"): at every grid point i, u itself and, for
every grid dimension (time first), its first and its second derivative.  With
D grid dimensions that is V = 1 + 2D unknowns per point, ordered
    v = 0: u,  v = 1 + 2d: du/dx_d,  v = 2 + 2d: d2u/dx_d2.
z is laid out [v][point], the point index running over the grid with the last
dimension fastest.  Keeping both derivatives in every dimension is what the
Taylor rows of Eqs. 6-7 need, and it reproduces the paper's variable counts
(5120 for a 32x32 grid, ~220k for 32^3: Section 3, "Scaling PDE Solving").

Rows, one family at a time (no row weights: the paper states none):
  E   (Eq. 3)  sum_v c_{v,i} z_{v,i} = b_i                     every point
  D1  (Eq. 5)  s_d z_{1+2d,i} - sum_j w_j u_{i+j e_d} = 0      every point, dim d
  D2  (Eq. 5)  s_d^2 z_{2+2d,i} - sum_j w_j u_{i+j e_d} = 0    every point, dim d
  TF  (Eq. 6)  u_i + s_d z_{1+2d,i} + s_d^2/2 z_{2+2d,i} - u_{next_d(i)} = 0
  TB  (Eq. 7)  u_i - s_d z_{1+2d,i} + s_d^2/2 z_{2+2d,i} - u_{prev_d(i)} = 0
  BC  (Eq. 4)  u_i = omega_i                                    i in the boundary set

Readings of points where the paper is silent or loose (each also listed in the
design notes):
  * Derivative rows sit at every grid point, boundary points included; this is
    what reproduces the paper's constraint counts (9212 for 32x32, ~420k for
    32^3).  Eq. 5 writes the second-difference form; first derivatives use the
    matching central form s u' = (u_{i+1} - u_{i-1}) / 2.
  * `stencil` 3 (default) or 5.  The paper says five-point central differences
    are used in practice with one-sided differences at the grid edges, while its
    worked example is the three-point form.  Five-point weights:
    s u' = (u_{-2} - 8 u_{-1} + 8 u_{+1} - u_{+2}) / 12,
    s^2 u'' = (-u_{-2} + 16 u_{-1} - 30 u_0 + 16 u_{+1} - u_{+2}) / 12,
    falling back to the three-point central form one point from an edge.
  * Edges of a non-periodic dimension use second-order one-sided three-point
    forms: s u'(0) = (-3 u_0 + 4 u_1 - u_2) / 2, s^2 u''(0) = u_0 - 2 u_1 + u_2,
    mirrored at the far edge (sign of the first derivative flipped).
  * Periodic dimensions wrap; they have no edges and every point has both a
    next and a previous neighbour.  Time is never periodic.
  * The boundary set B is the t = 0 face plus both faces of every non-periodic
    spatial dimension; `final_time_rows` adds the t = t_f face, which is what
    the paper's 32x32 count (9212 constraints) requires.  A corner point gets one
    boundary row.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

# Row family labels, in assembly order.
E, D1, D2, TF, TB, BC = 0, 1, 2, 3, 4, 5
FAMILY_NAMES = {E: "equation", D1: "first-derivative", D2: "second-derivative",
                TF: "taylor-forward", TB: "taylor-backward", BC: "boundary"}


def n_vars(ndim: int) -> int:
    return 1 + 2 * ndim


def first(d: int) -> int:
    return 1 + 2 * d


def second(d: int) -> int:
    return 2 + 2 * d


def multi_index(n):
    """(N, D) integer coordinates of every grid point, last dimension fastest."""
    axes = np.meshgrid(*[np.arange(k) for k in n], indexing="ij")
    return np.stack([a.ravel() for a in axes], axis=1)


def flat(idx, n):
    """Flat point index of (N, D) coordinates."""
    p = np.zeros(idx.shape[0], dtype=np.int64)
    for d, k in enumerate(n):
        p = p * k + idx[:, d]
    return p


def boundary_mask(geom):
    """Boolean mask over points of the boundary set B (Eq. 4 reading above)."""
    n = geom["n"]
    idx = multi_index(n)
    m = idx[:, 0] == 0
    if geom.get("final_time_rows", False):
        m |= idx[:, 0] == n[0] - 1
    for d in range(1, len(n)):
        if not geom["periodic"][d]:
            m |= (idx[:, d] == 0) | (idx[:, d] == n[d] - 1)
    return m


def _derivative_stencil(order, stencil, pos, n, periodic):
    """(offsets, weights) of the difference form of Eq. 5 for a point at
    coordinate `pos` of a dimension with `n` points.  The row reads
    s^order * z_deriv = sum_j weights[j] * u[pos + offsets[j]]."""
    c3 = {1: ([-1, 1], [-0.5, 0.5]), 2: ([-1, 0, 1], [1.0, -2.0, 1.0])}
    c5 = {1: ([-2, -1, 1, 2], [1 / 12, -8 / 12, 8 / 12, -1 / 12]),
          2: ([-2, -1, 0, 1, 2], [-1 / 12, 16 / 12, -30 / 12, 16 / 12, -1 / 12])}
    left = {1: ([0, 1, 2], [-1.5, 2.0, -0.5]), 2: ([0, 1, 2], [1.0, -2.0, 1.0])}
    right = {1: ([-2, -1, 0], [0.5, -2.0, 1.5]), 2: ([-2, -1, 0], [1.0, -2.0, 1.0])}
    if periodic:
        return (c5 if stencil == 5 else c3)[order]
    if pos == 0:
        return left[order]
    if pos == n - 1:
        return right[order]
    if stencil == 5 and 2 <= pos <= n - 3:
        return c5[order]
    return c3[order]


class _Rows:
    """Accumulates COO triplets and the right-hand side, row by row family."""

    def __init__(self, nv_total):
        self.r, self.c, self.v, self.d, self.kind = [], [], [], [], []
        self.nrows = 0
        self.ncols = nv_total

    def add(self, family, terms, rhs):
        """terms: list of (column array, value array) of equal length R; adds R
        rows whose entries are the given terms and whose rhs is `rhs`."""
        R = len(terms[0][0])
        rows = self.nrows + np.arange(R)
        for col, val in terms:
            self.r.append(rows)
            self.c.append(np.asarray(col, dtype=np.int64))
            self.v.append(np.broadcast_to(np.asarray(val, dtype=np.float64), (R,)))
        self.d.append(np.broadcast_to(np.asarray(rhs, dtype=np.float64), (R,)))
        self.kind.append(np.full(R, family, dtype=np.int8))
        self.nrows += R

    def build(self):
        A = sp.coo_matrix((np.concatenate(self.v), (np.concatenate(self.r),
                                                    np.concatenate(self.c))),
                          shape=(self.nrows, self.ncols)).tocsr()
        A.sum_duplicates()
        return A, np.concatenate(self.d).copy(), np.concatenate(self.kind)


def assemble(geom, coeff, b, omega, drop_zero_coeff=False):
    """Assemble one instance.

    geom   dict(n, step, periodic, stencil, final_time_rows)
    coeff  (V, N) per-point coefficients c_{v,i} of the equation rows (Eq. 3)
    b      (N,) right-hand side of the equation rows
    omega  (N,) Dirichlet values (read on boundary points only, Eq. 4)

    Returns (A, d, kind, owner): A is (n_c, V*N) CSR, d is (n_c,), kind labels
    each row with its family and owner gives the grid point that owns it.
    """
    n = tuple(geom["n"])
    D = len(n)
    V = n_vars(D)
    N = int(np.prod(n))
    steps = geom["step"]
    periodic = geom["periodic"]
    stencil = geom.get("stencil", 3)
    assert not periodic[0], "time is never periodic"
    assert stencil in (3, 5)
    for d in range(D):
        assert n[d] >= (5 if stencil == 5 else 3)
    coeff = np.asarray(coeff, dtype=np.float64).reshape(V, N)
    b = np.asarray(b, dtype=np.float64).reshape(N)
    omega = np.asarray(omega, dtype=np.float64).reshape(N)

    idx = multi_index(n)
    pts = np.arange(N)
    col = lambda v, p: v * N + p
    rows = _Rows(V * N)
    owners = []

    def neighbour(p_idx, d, off):
        q = p_idx.copy()
        q[:, d] = q[:, d] + off
        if periodic[d]:
            q[:, d] %= n[d]
        return flat(q, n)

    # Equation rows, Eq. 3: one per grid point.
    terms = []
    for v in range(V):
        if drop_zero_coeff and not np.any(coeff[v]):
            continue
        terms.append((col(v, pts), coeff[v]))
    rows.add(E, terms, b)
    owners.append(pts)

    # Derivative-consistency rows, Eq. 5: one per derivative unknown per point.
    for d in range(D):
        s = steps[d]
        for order, fam, var in ((1, D1, first(d)), (2, D2, second(d))):
            # group the points by their stencil (position class along dim d)
            classes = {}
            for pos in range(n[d]):
                offs, w = _derivative_stencil(order, stencil, pos, n[d], periodic[d])
                classes.setdefault((tuple(offs), tuple(w)), []).append(pos)
            for (offs, w), positions in classes.items():
                sel = np.isin(idx[:, d], positions)
                p = pts[sel]
                pi = idx[sel]
                t = [(col(var, p), s ** order)]
                for o, wj in zip(offs, w):
                    t.append((col(0, neighbour(pi, d, o)), -wj))
                rows.add(fam, t, 0.0)
                owners.append(p)

    # Taylor smoothness rows, Eqs. 6-7, in every dimension.
    for d in range(D):
        s = steps[d]
        for fam, sign in ((TF, 1.0), (TB, -1.0)):
            if periodic[d]:
                sel = np.ones(N, dtype=bool)
            elif sign > 0:
                sel = idx[:, d] < n[d] - 1
            else:
                sel = idx[:, d] > 0
            p = pts[sel]
            pi = idx[sel]
            t = [(col(0, p), 1.0),
                 (col(first(d), p), sign * s),
                 (col(second(d), p), 0.5 * s * s),
                 (col(0, neighbour(pi, d, int(sign))), -1.0)]
            rows.add(fam, t, 0.0)
            owners.append(p)

    # Initial / boundary rows, Eq. 4 (Dirichlet).
    p = pts[boundary_mask(geom)]
    rows.add(BC, [(col(0, p), 1.0)], omega[p])
    owners.append(p)

    A, dvec, kind = rows.build()
    return A, dvec, kind, np.concatenate(owners)


def counts(geom):
    """(n_v, n_c) of the assembled system without building it."""
    n = tuple(geom["n"])
    D = len(n)
    N = int(np.prod(n))
    nc = N                      # equation rows
    nc += 2 * D * N             # derivative rows
    for d in range(D):
        per = N if geom["periodic"][d] else N // n[d] * (n[d] - 1)
        nc += 2 * per           # forward + backward Taylor rows
    nc += int(boundary_mask(geom).sum())
    return n_vars(D) * N, nc
