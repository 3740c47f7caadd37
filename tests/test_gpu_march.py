"""Parity of the t-marching fused step with the FP64 oracle (fused_step = 4
puts it on every level it serves; 3, on the levels with enough columns).

The marching kernel serves levels with periodic x and y, n_x % 16 == 0
(columns of 16 x-rows) or n_x % 8 == 0 (8 rows), n_y % 64 == 0 and n_t % 8 == 0 in the transport layout (fields on c_x, c_y)
and the reaction-diffusion layout with c_xx = c_yy one field.  The cases
cover one and several columns in x and in y, rows of exactly 64 points (the
y halo wraps on both sides of one column), chunks of the time extent (the
warm-up planes of a chunk that starts inside the domain) and the one-sided
rows of the first and last plane.  Tolerances as in the other parity tests:
reduced operator 2e-5, forward z and adjoint d_z 1e-6 relative L2.
"""
import numpy as np
import pytest
import torch

from oracle import assemble as asm
from oracle import grad as og
from oracle import solve as osv
from paper_2502_18377_b300 import workloads as wl

pytestmark = pytest.mark.gpu

FWD_TOL = 1e-6
OP_TOL = 2e-5


def _round(w):
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


CASES = [
    # one column per instance: x wraps inside the column, y rows of 64
    ("transport_1col", lambda: wl.transport_2d(batch=2, n=(8, 16, 64))),
    # two columns in x, two chunks of 8 planes
    ("transport_2x_chunks", lambda: wl.transport_2d(batch=2, n=(16, 32, 64))),
    # two columns in y (64-point y halos inside the domain and across the wrap)
    ("transport_2y", lambda: wl.transport_2d(batch=1, n=(8, 16, 128))),
    ("reaction_diffusion_1col", lambda: wl.reaction_diffusion_2d(batch=2, n=(8, 16, 64))),
    ("reaction_diffusion_chunks", lambda: wl.reaction_diffusion_2d(batch=1, n=(16, 16, 128))),
    # columns of 8 x-rows (n_x not a multiple of 16): one column, three
    # columns with chunks
    ("transport_8rows", lambda: wl.transport_2d(batch=2, n=(8, 8, 64))),
    ("transport_8rows_3x_chunks", lambda: wl.transport_2d(batch=1, n=(16, 24, 64))),
    ("reaction_diffusion_8rows", lambda: wl.reaction_diffusion_2d(batch=1, n=(16, 8, 128))),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_marching_step_matches_oracle(name, make):
    """The reduced operator, the forward solve and the adjoint solve with the
    marching step meet the oracle; the operator agrees with the tile kernels'."""
    w = _round(make())
    s = _solver(w, fused_step=4)
    s_ref = _solver(w, fused_step=1)
    rng = np.random.default_rng(91)
    V, N = asm.n_vars(w.ndim), w.npoints
    u = rng.normal(size=(w.batch, N)).astype(np.float32)
    q = s.apply_reduced(_dev(w.fields), _dev(w.scalars), _dev(u)).cpu().numpy()
    q_ref = s_ref.apply_reduced(_dev(w.fields), _dev(w.scalars), _dev(u)).cpu().numpy()
    args = (_dev(w.fields), _dev(w.scalars), _dev(w.rhs), _dev(w.omega))
    z = s.forward(*args)
    g = rng.normal(size=(w.batch, V, N)).astype(np.float32)
    _, _, _, _, dz = s.adjoint(*args, z, _dev(g), reuse_setup=True, want_dz=True)
    z, dz = z.cpu().numpy(), dz.cpu().numpy()
    for b in range(w.batch):
        c = w.full_coeff()[:, b]
        A, d, kind, owner = asm.assemble(w.geom, c, w.rhs[b], w.omega[b])
        zr, lam, el = osv.solve_lsq_elim(A, d, V)
        ref = el.S @ u[b].astype(np.float64)
        assert _rel(q[b], ref) <= OP_TOL, (name, b, _rel(q[b], ref))
        assert _rel(q[b], q_ref[b]) <= OP_TOL, (name, b, _rel(q[b], q_ref[b]))
        assert _rel(z[b].ravel(), zr) <= FWD_TOL, (name, b, _rel(z[b].ravel(), zr), s.last_stats)
        dzr, _ = og.adjoint_elim(el, g[b].astype(np.float64).ravel())
        assert _rel(dz[b].ravel(), dzr) <= FWD_TOL, (name, b, _rel(dz[b].ravel(), dzr))


def test_marching_step_is_deterministic():
    """Two forward solves with the marching step give the same bits (the
    partial sums of every CTA are finished in a fixed order)."""
    w = _round(wl.transport_2d(batch=2, n=(16, 32, 64)))
    s = _solver(w, fused_step=4)
    args = (_dev(w.fields), _dev(w.scalars), _dev(w.rhs), _dev(w.omega))
    z1 = s.forward(*args).cpu().numpy()
    z2 = s.forward(*args).cpu().numpy()
    assert np.array_equal(z1, z2)


def test_marching_kernel_runs():
    """fused_step = 4 puts the marching kernel on the finest level of a
    qualifying problem, and fused_step = 1 does not."""
    from torch.profiler import ProfilerActivity, profile
    w = _round(wl.transport_2d(batch=2, n=(8, 32, 64)))
    u = _dev(np.random.default_rng(92).normal(size=(w.batch, w.npoints)))
    names = {}
    for fs in (1, 4):
        s = _solver(w, fused_step=fs)
        with profile(activities=[ProfilerActivity.CUDA]) as prof:
            s.apply_reduced(_dev(w.fields), _dev(w.scalars), u)
            torch.cuda.synchronize()
        names[fs] = " ".join(e.key for e in prof.key_averages())
    assert "k_march" in names[4], names[4]
    assert "k_march" not in names[1], names[1]
