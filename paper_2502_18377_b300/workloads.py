"""Seeded synthetic inputs for the batched linear-PDE least-squares solve.

This module only draws and lays out input data (coefficient fields, right-hand
sides, initial/boundary values, loss targets).  It holds none of the solver's
arithmetic, so both the CUDA path and the CPU oracle can take their inputs from
it without sharing any method code.

Every instance b of a workload with id `cfg` draws from
``numpy.random.default_rng(1000 * cfg + b)`` (plus a fixed offset per purpose),
so the same arrays can be regenerated on any machine.

The PDE family is Eq. 1 of the paper: sum_m c_m(t,x) u_m = b(t,x) on a regular
(t, x[, y]) grid, with Dirichlet data omega on the initial face (and on the
faces of non-periodic spatial dimensions).

Variable order per grid point (V = 1 + 2D for D grid dimensions):
    v = 0           u
    v = 1 + 2d      first derivative along dimension d   (d = 0 is time)
    v = 2 + 2d      second derivative along dimension d
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


def n_vars(ndim: int) -> int:
    return 1 + 2 * ndim


@dataclasses.dataclass
class Workload:
    """One batch of PDE instances.

    geom      dict(n=(n_t, n_x[, n_y]), step=(s_t, s_x[, s_y]),
                   periodic=(False, p_x[, p_y]), stencil=3|5,
                   final_time_rows=False)
    field_of  per variable v: index f of the coefficient field c_v reads, or -1
              when c_v is a per-instance scalar (several v may share one field)
    scalars   (V, B)  per-instance coefficient values for v with field_of[v] < 0
    fields    (F, B, N) coefficient fields, point index with the last dim fastest
    rhs       (B, N) right-hand side b of the equation rows
    omega     (B, N) Dirichlet values; only entries on boundary points are read
    target    (B, N) or None: u-target of the MSE loss used for adjoint solves
    """

    name: str
    geom: dict
    field_of: list
    scalars: np.ndarray
    fields: np.ndarray
    rhs: np.ndarray
    omega: np.ndarray
    target: np.ndarray | None = None

    @property
    def batch(self) -> int:
        return self.rhs.shape[0]

    @property
    def ndim(self) -> int:
        return len(self.geom["n"])

    @property
    def npoints(self) -> int:
        return int(np.prod(self.geom["n"]))

    def full_coeff(self) -> np.ndarray:
        """(V, B, N) float64 per-point coefficients (layout expansion only)."""
        V, B, N = n_vars(self.ndim), self.batch, self.npoints
        out = np.empty((V, B, N))
        for v in range(V):
            f = self.field_of[v]
            out[v] = self.fields[f] if f >= 0 else self.scalars[v][:, None]
        return out


def _geom(n, step, periodic, stencil=3, final_time_rows=False):
    return dict(n=tuple(int(k) for k in n), step=tuple(float(s) for s in step),
                periodic=tuple(bool(p) for p in periodic), stencil=int(stencil),
                final_time_rows=bool(final_time_rows))


def _coords(n, periodic, lengths):
    """Grid coordinates per dimension: non-periodic [0, L] with n points
    (step L/(n-1)), periodic [0, L) with n points (step L/n)."""
    out, steps = [], []
    for k, p, L in zip(n, periodic, lengths):
        s = L / k if p else L / (k - 1)
        out.append(np.arange(k) * s)
        steps.append(s)
    return out, steps


def smooth_field(rng, coords, lo, hi, modes=8):
    """Sum of `modes` random low-frequency cosines on the grid, mapped affinely
    so that its min is `lo` and its max is `hi`.  coords[0] is time (k_t/2 cycles
    over [0, 1]); the other coordinates are on [0, 1) with integer wavenumbers."""
    mesh = np.meshgrid(*coords, indexing="ij")
    acc = np.zeros(mesh[0].shape)
    for _ in range(modes):
        kt = rng.integers(0, 3)
        ks = rng.integers(0, 4, size=len(coords) - 1)
        amp = rng.normal()
        theta = rng.uniform(0.0, 2.0 * math.pi)
        phase = kt / 2.0 * mesh[0]
        for kk, m in zip(ks, mesh[1:]):
            phase = phase + kk * m
        acc += amp * np.cos(2.0 * math.pi * phase + theta)
    mn, mx = acc.min(), acc.max()
    if mx - mn < 1e-12:
        return np.full(acc.shape, 0.5 * (lo + hi))
    return lo + (hi - lo) * (acc - mn) / (mx - mn)


def box_filter(x, periodic):
    """Separable 3-point box filter; wraps in periodic dims, replicates edges
    otherwise."""
    y = x
    for ax, p in enumerate(periodic):
        if p:
            y = (np.roll(y, 1, ax) + y + np.roll(y, -1, ax)) / 3.0
        else:
            pad = [(0, 0)] * y.ndim
            pad[ax] = (1, 1)
            yp = np.pad(y, pad, mode="edge")
            sl = lambda a, b: tuple(slice(a, b) if i == ax else slice(None)
                                    for i in range(y.ndim))
            y = (yp[sl(0, -2)] + yp[sl(1, -1)] + yp[sl(2, None)]) / 3.0
    return y


def low_mode_field(rng, geom, modes=4):
    """Sum of `modes` products of a random quadratic in t and a random
    lowest-wavenumber cosine (wavenumbers 0..2 per spatial dimension, over the
    grid's extent) with N(0, 1) amplitudes: a smooth grid function (N,) used
    as a manufactured solution."""
    n = tuple(geom["n"])
    coords = [np.arange(k) / (k - 1 if (d == 0 or not geom["periodic"][d]) else k)
              for d, k in enumerate(n)]
    mesh = np.meshgrid(*coords, indexing="ij")
    acc = np.zeros(mesh[0].shape)
    for _ in range(modes):
        a = rng.normal(size=3)
        ks = rng.integers(0, 3, size=len(n) - 1)
        phase = rng.uniform(0.0, 2.0 * math.pi)
        arg = phase + sum(2.0 * math.pi * k * m for k, m in zip(ks, mesh[1:]))
        acc += rng.normal() * (a[0] + a[1] * mesh[0] + a[2] * mesh[0] ** 2) * np.cos(arg)
    return acc.ravel()


def advection_diffusion_1d(batch=4, n=(32, 32), seed_base=1000, stencil=3,
                           final_time_rows=False):
    """u_t + a u_x - nu u_xx = f on t in [0,1], x in [0,1] (Dirichlet in x).

    Manufactured solution u = sin(2 pi k x) exp(-t), k = 1 + (b mod 2);
    a ~ U[-1, 1], nu ~ U[0.01, 0.1] per instance (scalar coefficients);
    f follows from u analytically; omega = u."""
    (t, x), steps = _coords(n, (False, False), (1.0, 1.0))
    T, X = np.meshgrid(t, x, indexing="ij")
    V, N = 5, n[0] * n[1]
    scal = np.zeros((V, batch))
    rhs = np.empty((batch, N))
    om = np.empty((batch, N))
    for b in range(batch):
        rng = np.random.default_rng(seed_base + b)
        a = rng.uniform(-1.0, 1.0)
        nu = rng.uniform(0.01, 0.1)
        k = 1 + b % 2
        w = 2.0 * math.pi * k
        u = np.sin(w * X) * np.exp(-T)
        f = -u + a * w * np.cos(w * X) * np.exp(-T) + nu * w * w * u
        scal[:, b] = [0.0, 1.0, 0.0, a, -nu]
        rhs[b] = f.ravel()
        om[b] = u.ravel()
    return Workload("advection_diffusion_1d", _geom(n, steps, (False, False), stencil,
                                                    final_time_rows),
                    [-1] * V, scal, np.zeros((0, batch, N)), rhs, om)


def reaction_diffusion_2d(batch=16, n=(32, 64, 64), seed_base=2000, stencil=3):
    """u_t = d(t,x,y) (u_xx + u_yy) + r(t,x,y) u + f, periodic in x and y.

    d in [0.01, 0.1] and r in [-1, 1] are smooth seeded fields; f ~ N(0,1)
    smoothed by a 3-point box filter; u(0, .) = 0.  Written as
    u_t - d u_xx - d u_yy - r u = f: field 0 = -d (shared by u_xx and u_yy),
    field 1 = -r (on u).  The loss target is a smoothed N(0, 1) field."""
    periodic = (False, True, True)
    coords, steps = _coords(n, periodic, (1.0, 1.0, 1.0))
    V, N = 7, int(np.prod(n))
    fields = np.empty((2, batch, N))
    rhs = np.empty((batch, N))
    tgt = np.empty((batch, N))
    for b in range(batch):
        rng = np.random.default_rng(seed_base + b)
        d = smooth_field(rng, coords, 0.01, 0.1)
        r = smooth_field(rng, coords, -1.0, 1.0)
        f = box_filter(rng.normal(size=n), periodic)
        fields[0, b] = -d.ravel()
        fields[1, b] = -r.ravel()
        rhs[b] = f.ravel()
        rng_t = np.random.default_rng(seed_base + 500_000 + b)
        tgt[b] = box_filter(rng_t.normal(size=n), periodic).ravel()
    scal = np.zeros((V, batch))
    scal[1] = 1.0
    field_of = [1, -1, -1, -1, 0, -1, 0]
    return Workload("reaction_diffusion_2d", _geom(n, steps, periodic, stencil),
                    field_of, scal, fields, rhs, np.zeros((batch, N)), tgt)


def linearized_burgers_1d(batch=32, n=(128, 256), seed_base=3000, stencil=3):
    """u_t + c(t,x) u_x - 0.01 u_xx = 0, periodic in x.

    c is a smooth seeded field in [-1, 1]; u(0, x) = sum_j a_j sin(2 pi k_j x)
    with 4 distinct k_j in {1..8}, a_j ~ U[-1, 1].  The loss target is a
    smoothed N(0,1) field scaled by 0.1 (the MSE target is set by the caller
    when it wants it relative to a reference solution)."""
    periodic = (False, True)
    coords, steps = _coords(n, periodic, (1.0, 1.0))
    V, N = 5, n[0] * n[1]
    fields = np.empty((1, batch, N))
    om = np.zeros((batch, N))
    tgt = np.empty((batch, N))
    x = coords[1]
    for b in range(batch):
        rng = np.random.default_rng(seed_base + b)
        c = smooth_field(rng, coords, -1.0, 1.0)
        ks = rng.choice(np.arange(1, 9), size=4, replace=False)
        amps = rng.uniform(-1.0, 1.0, size=4)
        u0 = sum(a * np.sin(2.0 * math.pi * k * x) for a, k in zip(amps, ks))
        fields[0, b] = c.ravel()
        o = np.zeros(n)
        o[0, :] = u0
        om[b] = o.ravel()
        rng_t = np.random.default_rng(seed_base + 500_000 + b)
        tgt[b] = 0.1 * box_filter(rng_t.normal(size=n), periodic).ravel()
    scal = np.zeros((V, batch))
    scal[1] = 1.0
    scal[4] = -0.01
    field_of = [-1, -1, -1, 0, -1]
    return Workload("linearized_burgers_1d", _geom(n, steps, periodic, stencil),
                    field_of, scal, fields, np.zeros((batch, N)), om, tgt)


def transport_2d(batch=4, n=(32, 256, 256), seed_base=5000, stencil=3):
    """u_t + v1 u_x + v2 u_y - 1e-3 (u_xx + u_yy) = sin(4 y) on [0, 2pi)^2.

    (v1, v2) = (d psi/dy, -d psi/dx) from a random stream function with
    |psi_hat(k)| ~ |k|^-3 for 1 <= |k| <= 85, scaled so max |v| = 1, steady in
    t; u(0, .) = 0."""
    periodic = (False, True, True)
    coords, steps = _coords(n, periodic, (1.0, 2.0 * math.pi, 2.0 * math.pi))
    V, N = 7, int(np.prod(n))
    nx, ny = n[1], n[2]
    kx = np.fft.fftfreq(nx, 1.0 / nx)[:, None]
    ky = np.fft.fftfreq(ny, 1.0 / ny)[None, :]
    kk = np.sqrt(kx ** 2 + ky ** 2)
    band = (kk >= 1.0) & (kk <= 85.0)
    fields = np.empty((2, batch, N))
    rhs = np.empty((batch, N))
    tgt = np.empty((batch, N))
    y = coords[2]
    for b in range(batch):
        rng = np.random.default_rng(seed_base + b)
        psi_hat = (rng.normal(size=(nx, ny)) + 1j * rng.normal(size=(nx, ny)))
        psi_hat = np.where(band, psi_hat * np.where(band, kk, 1.0) ** -3.0, 0.0)
        v1 = np.real(np.fft.ifft2(1j * ky * psi_hat))
        v2 = -np.real(np.fft.ifft2(1j * kx * psi_hat))
        vmax = np.sqrt(v1 ** 2 + v2 ** 2).max()
        v1, v2 = v1 / vmax, v2 / vmax
        fields[0, b] = np.broadcast_to(v1, n).ravel()
        fields[1, b] = np.broadcast_to(v2, n).ravel()
        rhs[b] = np.broadcast_to(np.sin(4.0 * y)[None, None, :], n).ravel()
        rng_t = np.random.default_rng(seed_base + 500_000 + b)
        tgt[b] = box_filter(rng_t.normal(size=n), periodic).ravel()
    scal = np.zeros((V, batch))
    scal[1] = 1.0
    scal[4] = -1e-3
    scal[6] = -1e-3
    field_of = [-1, -1, -1, 0, -1, 1, -1]
    return Workload("transport_2d", _geom(n, steps, periodic, stencil),
                    field_of, scal, fields, rhs, np.zeros((batch, N)), tgt)


def laplace_2d(batch=32, n=32, seed_base=6000, stencil=3):
    """Laplace's equation u_yy + u_xx = 0 on the unit square (the solver test
    of the paper's experiments section and its time / memory table, batch 32).

    The grid's first axis plays y: c_tt = c_xx = 1, every other coefficient 0
    (per-instance scalars), b = 0, Dirichlet rows on all four faces (the
    final-plane face included).  Boundary data and the reference solution come
    from the harmonic function u = sum_{k=1..3} a_k sin(k pi x) sinh(k pi y) /
    sinh(k pi), a_k ~ U[-1, 1] per instance: sinusoidal on the face y = 1,
    zero on the other three.  `target` holds u on the whole grid."""
    (y, x), steps = _coords((n, n), (False, False), (1.0, 1.0))
    Y, X = np.meshgrid(y, x, indexing="ij")
    V, N = 5, n * n
    scal = np.zeros((V, batch))
    scal[2] = 1.0
    scal[4] = 1.0
    om = np.empty((batch, N))
    for b in range(batch):
        rng = np.random.default_rng(seed_base + b)
        a = rng.uniform(-1.0, 1.0, size=3)
        u = sum(a[k - 1] * np.sin(k * math.pi * X) * np.sinh(k * math.pi * Y) / math.sinh(k * math.pi)
                for k in (1, 2, 3))
        om[b] = u.ravel()
    return Workload("laplace_2d", _geom((n, n), steps, (False, False), stencil, True),
                    [-1] * V, scal, np.zeros((0, batch, N)), np.zeros((batch, N)), om, om.copy())


def random_problem(seed, n, periodic, stencil=3, batch=1, final_time_rows=False,
                   lengths=None, field_all=True):
    """Generic random instance for property tests: every coefficient is a
    random field (c_t kept away from 0), random rhs and boundary values."""
    D = len(n)
    V = n_vars(D)
    lengths = lengths or (1.0,) * D
    _, steps = _coords(n, periodic, lengths)
    N = int(np.prod(n))
    rng = np.random.default_rng(seed)
    fields = rng.uniform(-1.0, 1.0, size=(V, batch, N))
    fields[1] = rng.uniform(0.5, 1.5, size=(batch, N))
    for d in range(1, D):
        fields[2 + 2 * d] = -rng.uniform(0.01, 0.1, size=(batch, N))
    rhs = rng.normal(size=(batch, N))
    om = rng.normal(size=(batch, N))
    tgt = rng.normal(size=(batch, N))
    field_of = list(range(V)) if field_all else [-1] * V
    scal = fields[:, :, 0].copy()
    return Workload("random", _geom(n, steps, periodic, stencil, final_time_rows),
                    field_of, scal, fields if field_all else np.zeros((0, batch, N)),
                    rhs, om, tgt)


CONFIGS = {
    1: advection_diffusion_1d,
    2: reaction_diffusion_2d,
    3: linearized_burgers_1d,
    4: lambda batch=8, n=(64, 128, 128), seed_base=4000, stencil=3:
        reaction_diffusion_2d(batch, n, seed_base, stencil),
    5: transport_2d,
}
