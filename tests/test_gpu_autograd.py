"""The NeuRLP-PDE layer as a torch.autograd.Function (solve + loss.backward)
against the oracle's gradients (Eq. 11 and the formulas after it)."""
import numpy as np
import pytest
import torch

from oracle import assemble as asm
from oracle import grad as og
from oracle import solve as osv
from paper_2502_18377_b300 import workloads as wl

pytestmark = pytest.mark.gpu
GRAD_TOL = 1e-5


def _round(w):
    r = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)
    return wl.Workload(w.name, w.geom, list(w.field_of), r(w.scalars), r(w.fields), r(w.rhs), r(w.omega),
                       None if w.target is None else r(w.target))


def _leaf(a):
    return torch.tensor(np.asarray(a, dtype=np.float32), device="cuda").contiguous().requires_grad_(True)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _oracle_grads(w, b, tgt):
    """Oracle gradients of l = mean over (b, i) of (u - target)^2."""
    V, N, B = asm.n_vars(w.ndim), w.npoints, w.batch
    A, d, kind, owner = asm.assemble(w.geom, w.full_coeff()[:, b], w.rhs[b], w.omega[b])
    z, lam, el = osv.solve_lsq_elim(A, d, V)
    g = np.zeros(V * N)
    g[:N] = 2.0 * (z[:N] - tgt[b]) / (N * B)
    dz, dlam = og.adjoint_elim(el, g)
    dc, db, dw = og.gradients(w.geom, A, d, kind, owner, z, lam, dz, dlam)
    return dc, db, dw


def _check(w, fields, scal, rhs, om, tgt):
    F = w.fields.shape[0]
    V = asm.n_vars(w.ndim)
    gf, gs, gr, go = (t.grad.cpu().numpy() for t in (fields, scal, rhs, om))
    for b in range(w.batch):
        dc, db, dw = _oracle_grads(w, b, tgt)
        for f in range(F):
            ref = sum(dc[v] for v in range(V) if w.field_of[v] == f)
            assert _rel(gf[f, b], ref) <= GRAD_TOL, (b, f, _rel(gf[f, b], ref))
        for v in range(V):
            if w.field_of[v] < 0:
                assert abs(gs[v, b] - dc[v].sum()) <= GRAD_TOL * max(1.0, np.abs(dc[v]).sum())
        assert _rel(gr[b], db) <= GRAD_TOL
        assert _rel(go[b], dw) <= GRAD_TOL


@pytest.mark.parametrize("recompute", [False, True])
def test_autograd_backward_matches_oracle(recompute):
    from paper_2502_18377_b300.autograd import solve
    from paper_2502_18377_b300.binding import Solver
    w = _round(wl.reaction_diffusion_2d(batch=2, n=(8, 16, 16)))
    s = Solver(w.geom, w.batch, w.field_of, w.fields.shape[0])
    fields, scal, rhs, om = (_leaf(a) for a in (w.fields, w.scalars, w.rhs, w.omega))
    tgt = torch.tensor(np.asarray(w.target, dtype=np.float32), device="cuda")
    z = solve(fields, scal, rhs, om, s, recompute=recompute)
    loss = ((z[:, 0] - tgt) ** 2).mean()
    g0 = s.generation()
    loss.backward()
    # the kept state is reused unless asked to recompute (one more forward)
    assert s.generation() == g0 + (1 if recompute else 0)
    _check(w, fields, scal, rhs, om, w.target)


def test_autograd_with_an_intervening_forward():
    """Another forward on the same solver between this forward and its
    backward (other data): the backward pass sees the changed generation and
    recomputes, so its gradients are still those of its own data."""
    from paper_2502_18377_b300.autograd import solve
    from paper_2502_18377_b300.binding import Solver
    w = _round(wl.reaction_diffusion_2d(batch=2, n=(8, 16, 16)))
    w2 = _round(wl.reaction_diffusion_2d(batch=2, n=(8, 16, 16), seed_base=9000))
    s = Solver(w.geom, w.batch, w.field_of, w.fields.shape[0])
    fields, scal, rhs, om = (_leaf(a) for a in (w.fields, w.scalars, w.rhs, w.omega))
    tgt = torch.tensor(np.asarray(w.target, dtype=np.float32), device="cuda")
    z = solve(fields, scal, rhs, om, s)
    loss = ((z[:, 0] - tgt) ** 2).mean()
    with torch.no_grad():
        other = [torch.tensor(np.asarray(a, dtype=np.float32), device="cuda") for a in
                 (w2.fields, w2.scalars, w2.rhs, w2.omega)]
        s.forward(*other)
    g0 = s.generation()
    loss.backward()
    assert s.generation() == g0 + 1          # recomputed
    _check(w, fields, scal, rhs, om, w.target)


def test_adjoint_reuse_with_other_buffers_recomputes():
    """MPN_REUSE_SETUP with input buffers other than the last forward's: the
    library recomputes the forward instead of using the kept state."""
    from paper_2502_18377_b300.binding import Solver
    w = _round(wl.reaction_diffusion_2d(batch=2, n=(8, 16, 16)))
    s = Solver(w.geom, w.batch, w.field_of, w.fields.shape[0])
    dev = lambda a: torch.tensor(np.asarray(a, dtype=np.float32), device="cuda").contiguous()
    args = (dev(w.fields), dev(w.scalars), dev(w.rhs), dev(w.omega))
    z = s.forward(*args)
    g = torch.zeros((w.batch, 7, w.npoints), device="cuda")
    g[:, 0] = 1.0
    g0 = s.generation()
    s.adjoint(*args, z, g, reuse_setup=True)
    assert s.generation() == g0
    copies = tuple(a.clone() for a in args)
    s.adjoint(*copies, z, g, reuse_setup=True)
    assert s.generation() == g0 + 1
