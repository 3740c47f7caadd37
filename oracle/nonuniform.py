"""Constraint system with per-interval steps and Neumann / mixed boundary
rows (Section 2 "discretization" and boundary types; Section 3, Eqs. 3-8),
and the gradient of the loss with respect to every interval (the learnable
steps), in FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Grid: along dimension d the points x_0 < ... < x_{n-1} are separated by the
intervals h_k = x_{k+1} - x_k (k < n - 1; a periodic dimension has a
further interval h_{n-1} closing the period).  Rows, with the readings below:

  E   (Eq. 3)   sum_v c_{v,i} z_{v,i} = b_i                      every point
  D1  (Eq. 5)   sbar_i z_{1+2d,i} - sum_j w1_j u_{i+j} = 0       every point
  D2  (Eq. 5)   sbar_i^2 z_{2+2d,i} - sum_j w2_j u_{i+j} = 0     every point
  TF  (Eq. 6)   u_i + h_i z_{1+2d,i} + h_i^2/2 z_{2+2d,i} - u_{i+1} = 0
  TB  (Eq. 7)   u_i - h_{i-1} z_{1+2d,i} + h_{i-1}^2/2 z_{2+2d,i} - u_{i-1} = 0
  BC  (Eq. 4 and its Neumann / mixed kinds)
                alpha u_i + beta z_{1+2d,i} = omega_i            boundary points

Readings where the paper is silent:
  * Derivative rows with unequal intervals: the three-point forms exact for
    quadratics (central inside, one-sided at the edges of a non-periodic
    dimension), in the multiplied form of Eq. 5 with the local step
    sbar_i = (h_{i-1} + h_i) / 2 inside and the adjacent interval at an edge.
    With equal intervals every row is that of the uniform assembly.
  * Boundary kinds per spatial dimension, both faces alike: Dirichlet
    (alpha = 1, beta = 0, the default), Neumann (alpha = 0, beta = 1) or mixed
    (both nonzero), on the derivative along that dimension.  The t = 0 face
    (and the t = t_f face with final_time_rows) is Dirichlet.  A point on
    several faces gets one row, of the first face in the order t = 0,
    t = t_f, then spatial dimensions in order, lower face first.
  * Gradients with respect to the intervals follow the gradient formula
    after Eq. 11: dl/dh_k = sum over the entries of A of
    (d_lambda z*^T + lambda* d_z^T) times d(entry)/dh_k; d does not depend on
    the steps.  The entries are written as float64 torch expressions of the
    intervals, so d(entry)/dh_k comes from automatic differentiation.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import torch

from . import assemble as asm


def uniform_intervals(geom):
    """Per-dimension interval arrays of a uniform geometry (dict with `step`)."""
    out = []
    for d, n in enumerate(geom["n"]):
        m = n if geom["periodic"][d] else n - 1
        out.append(np.full(m, float(geom["step"][d])))
    return out


def _dim_forms(n, h, periodic):
    """Difference forms along one dimension: for each order (1, 2) a list of
    (offset, weight tensor [n]) and the scale tensor sbar [n] of the row
    sbar^order z = sum_j weight_j u_{i+j}.  h: interval tensor."""
    idx = torch.arange(n)
    if periodic:
        hm = h[(idx - 1) % n]
        hp = h[idx]
    else:
        hm = torch.cat([h[:1], h])                       # h_{i-1}; index 0 unused
        hp = torch.cat([h, h[-1:]])                      # h_i; index n-1 unused
    sbar = 0.5 * (hm + hp)
    # central forms (exact for quadratics)
    c1 = {-1: -hp / (hm * (hm + hp)), 0: (hp - hm) / (hm * hp), 1: hm / (hp * (hm + hp))}
    c2 = {-1: 2.0 / (hm * (hm + hp)), 0: -2.0 / (hm * hp), 1: 2.0 / (hp * (hm + hp))}
    w1 = {o: torch.zeros(n, dtype=h.dtype) for o in (-2, -1, 0, 1, 2)}
    w2 = {o: torch.zeros(n, dtype=h.dtype) for o in (-2, -1, 0, 1, 2)}
    scale = sbar.clone()
    inner = torch.ones(n, dtype=torch.bool)
    if not periodic:
        inner[0] = inner[-1] = False
    for o in (-1, 0, 1):
        w1[o] = torch.where(inner, sbar * c1[o], w1[o])
        w2[o] = torch.where(inner, sbar * sbar * c2[o], w2[o])
    if not periodic:
        a, b = h[0], h[1]                                # first point: intervals to the right
        f1 = {0: -(2 * a + b) / (a * (a + b)), 1: (a + b) / (a * b), 2: -a / (b * (a + b))}
        f2 = {0: 2.0 / (a * (a + b)), 1: -2.0 / (a * b), 2: 2.0 / (b * (a + b))}
        g, q = h[-1], h[-2]                              # last point: intervals to the left
        l1 = {0: (2 * g + q) / (g * (g + q)), -1: -(g + q) / (g * q), -2: g / (q * (g + q))}
        l2 = {0: 2.0 / (g * (g + q)), -1: -2.0 / (g * q), -2: 2.0 / (q * (g + q))}
        first = idx == 0
        last = idx == n - 1
        scale = torch.where(first, a, torch.where(last, g, scale))
        for o in (0, 1, 2):
            w1[o] = torch.where(first, a * f1[o], w1[o])
            w2[o] = torch.where(first, a * a * f2[o], w2[o])
        for o in (0, -1, -2):
            w1[o] = torch.where(last, g * l1[o], w1[o])
            w2[o] = torch.where(last, g * g * l2[o], w2[o])
    return {1: w1, 2: w2}, scale, hm, hp


def _bc_rows(geom, idx):
    """Boundary points and, per point, (alpha, beta, dim) of its row."""
    n = geom["n"]
    D = len(n)
    bc = geom.get("bc", {})
    N = idx.shape[0]
    taken = np.zeros(N, dtype=bool)
    pts, alpha, beta, dim = [], [], [], []

    def add(mask, a, bt, d):
        sel = mask & ~taken
        p = np.flatnonzero(sel)
        pts.append(p)
        alpha.append(np.full(p.size, float(a)))
        beta.append(np.full(p.size, float(bt)))
        dim.append(np.full(p.size, d, dtype=np.int64))
        taken[sel] = True

    add(idx[:, 0] == 0, 1.0, 0.0, 0)
    if geom.get("final_time_rows", False):
        add(idx[:, 0] == n[0] - 1, 1.0, 0.0, 0)
    for d in range(1, D):
        if geom["periodic"][d]:
            continue
        a, bt = bc.get(d, (1.0, 0.0))
        add(idx[:, d] == 0, a, bt, d)
        add(idx[:, d] == n[d] - 1, a, bt, d)
    return (np.concatenate(pts), np.concatenate(alpha), np.concatenate(beta), np.concatenate(dim))


def entries(geom, coeff, b, omega, intervals):
    """COO triplets of A (values as float64 torch expressions of the interval
    tensors), d, row family and owning point of every row.

    intervals: per dimension a 1-D float64 tensor (n - 1 entries, n when
    periodic).  geom may carry bc = {dim: (alpha, beta)}."""
    if geom.get("stencil", 3) != 3:
        raise ValueError("per-interval steps take the three-point forms only")
    n = tuple(geom["n"])
    D = len(n)
    V = asm.n_vars(D)
    N = int(np.prod(n))
    coeff = np.asarray(coeff, dtype=np.float64).reshape(V, N)
    b = np.asarray(b, dtype=np.float64).reshape(N)
    omega = np.asarray(omega, dtype=np.float64).reshape(N)
    idx = asm.multi_index(n)
    pts = np.arange(N)
    R, C, Vals, dv, kind, owner = [], [], [], [], [], []
    nrow = 0

    def add(family, terms, rhs, own):
        nonlocal nrow
        rows = nrow + np.arange(own.size)
        for col, val in terms:
            R.append(rows)
            C.append(np.asarray(col, dtype=np.int64))
            Vals.append(val if torch.is_tensor(val) else torch.as_tensor(np.broadcast_to(val, own.shape).copy()))
        dv.append(np.broadcast_to(np.asarray(rhs, dtype=np.float64), own.shape))
        kind.append(np.full(own.size, family, dtype=np.int8))
        owner.append(own)
        nrow += own.size

    def nbr(d, off):
        q = idx.copy()
        q[:, d] += off
        if geom["periodic"][d]:
            q[:, d] %= n[d]
        return asm.flat(q, n)

    # equation rows (Eq. 3)
    add(asm.E, [(v * N + pts, coeff[v]) for v in range(V)], b, pts)
    # derivative rows (Eq. 5) and Taylor rows (Eqs. 6-7) per dimension
    for d in range(D):
        h = intervals[d]
        forms, scale, hm, hp = _dim_forms(n[d], h, geom["periodic"][d])
        pos = torch.as_tensor(idx[:, d])
        for order, fam, var in ((1, asm.D1, asm.first(d)), (2, asm.D2, asm.second(d))):
            terms = [(var * N + pts, scale[pos] ** order)]
            w = forms[order]
            for o in (-2, -1, 0, 1, 2):
                wo = w[o][pos]
                ok = np.asarray((wo != 0).detach().numpy())
                if not ok.any():
                    continue
                q = idx.copy()
                q[:, d] = q[:, d] + o
                if geom["periodic"][d]:
                    q[:, d] %= n[d]
                q[:, d] = np.clip(q[:, d], 0, n[d] - 1)
                terms.append((asm.flat(q, n), -wo))
            add(fam, terms, 0.0, pts)
        per = geom["periodic"][d]
        fwd = np.ones(N, dtype=bool) if per else idx[:, d] < n[d] - 1
        bwd = np.ones(N, dtype=bool) if per else idx[:, d] > 0
        for fam, sel, sign in ((asm.TF, fwd, 1.0), (asm.TB, bwd, -1.0)):
            p = pts[sel]
            s = (hp if sign > 0 else hm)[torch.as_tensor(idx[sel, d])]
            add(fam, [(p, 1.0), (asm.first(d) * N + p, sign * s), (asm.second(d) * N + p, 0.5 * s * s),
                      (nbr(d, int(sign))[sel], -1.0)], 0.0, p)
    # boundary rows (Eq. 4, Neumann, mixed)
    p, al, bt, dm = _bc_rows(geom, idx)
    terms = [(p, al)]
    dcol = np.where(dm > 0, (1 + 2 * dm) * N + p, p)
    terms.append((dcol, np.where(dm > 0, bt, 0.0)))
    add(asm.BC, terms, omega[p], p)
    rows = np.concatenate(R)
    cols = np.concatenate(C)
    vals = torch.cat([v.reshape(-1).to(torch.float64) for v in Vals])
    return rows, cols, vals, np.concatenate(dv), np.concatenate(kind), np.concatenate(owner), nrow, V * N


def assemble(geom, coeff, b, omega, intervals=None):
    """(A, d, kind, owner) as scipy CSR with the given per-interval steps
    (numpy arrays; the uniform steps of geom when None)."""
    iv = [torch.as_tensor(np.asarray(h, dtype=np.float64)) for h in (intervals or uniform_intervals(geom))]
    rows, cols, vals, d, kind, owner, nr, nc = entries(geom, coeff, b, omega, iv)
    A = sp.coo_matrix((vals.detach().numpy(), (rows, cols)), shape=(nr, nc)).tocsr()
    A.sum_duplicates()
    A.eliminate_zeros()
    return A, d, kind, owner


def step_gradients(geom, coeff, b, omega, intervals, z, lam, dz, dlam):
    """dl/dh for every interval of every dimension: the entries of
    d_lambda z*^T + lambda* d_z^T (the gradient formula after Eq. 11) times the
    derivative of each entry of A with respect to the intervals."""
    iv = [torch.tensor(np.asarray(h, dtype=np.float64), requires_grad=True) for h in intervals]
    rows, cols, vals, *_ = entries(geom, coeff, b, omega, iv)
    dA = np.asarray(dlam)[rows] * np.asarray(z)[cols] + np.asarray(lam)[rows] * np.asarray(dz)[cols]
    total = (vals * torch.as_tensor(dA)).sum()
    grads = torch.autograd.grad(total, iv, allow_unused=True)
    return [g.numpy() if g is not None else np.zeros(len(h)) for g, h in zip(grads, intervals)]
