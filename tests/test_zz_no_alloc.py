"""The allocation-free operator apply against the regular one.

mpn_apply_reduced_noalloc exists for callers that cannot allocate device
memory (their device memory belongs to another allocator, or allocation is
not acceptable on their path).  It must give the same q = S u as
mpn_apply_reduced, which runs on the problem's own workspace; both are FP32
applies of the same operator, compared at the tolerance the operator parity
test uses.  Two calls in a row check that the shared scratch array carries
nothing over from one call to the next.  This file is collected last.
"""
import numpy as np
import pytest
import torch

from paper_2502_18377_b300 import workloads as wl

pytestmark = pytest.mark.gpu
TOL = 2e-5


def _dev(a):
    return torch.tensor(np.asarray(a, dtype=np.float32), device="cuda").contiguous()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("make", [
    lambda: wl.reaction_diffusion_2d(batch=3, n=(8, 16, 16)),
    lambda: wl.random_problem(41, (9, 20), (False, False), batch=2, final_time_rows=True),
    lambda: wl.random_problem(42, (6, 10, 12), (False, True, False), batch=2, field_all=False),
])
def test_noalloc_apply_matches_regular_apply(make):
    from paper_2502_18377_b300.binding import Solver, apply_reduced_noalloc, make_desc
    w = make()
    F = w.fields.shape[0]
    fields, scal = _dev(w.fields), _dev(w.scalars)
    s = Solver(w.geom, w.batch, w.field_of, F)
    desc = make_desc(w.geom, w.batch, w.field_of, F)
    rng = np.random.default_rng(0)
    q_na = torch.empty((w.batch, w.npoints), device="cuda")
    for call in range(2):
        u = _dev(rng.normal(size=(w.batch, w.npoints)))
        ref = s.apply_reduced(fields, scal, u).cpu().numpy()
        apply_reduced_noalloc(desc, fields, scal, u, q_na)
        torch.cuda.synchronize()
        got = q_na.cpu().numpy()
        for b in range(w.batch):
            assert _rel(got[b], ref[b]) <= TOL, (call, b, _rel(got[b], ref[b]))


def test_noalloc_rejects_oversize():
    from paper_2502_18377_b300.binding import NOALLOC_MAX_POINTS, MpnError, apply_reduced_noalloc, make_desc
    w = wl.reaction_diffusion_2d(batch=1, n=(8, 16, 16))
    geom = dict(w.geom)
    n_big = (8, 16, NOALLOC_MAX_POINTS // 128 + 16)
    geom["n"] = n_big
    geom["step"] = (1.0, 1.0, 1.0)
    desc = make_desc(geom, 1, w.field_of, 2)
    N = int(np.prod(n_big))
    u = torch.zeros(N, device="cuda")
    q = torch.zeros(N, device="cuda")
    fields = torch.zeros((2, 1, N), device="cuda")
    scal = torch.zeros((7, 1), device="cuda")
    with pytest.raises(MpnError) as e:
        apply_reduced_noalloc(desc, fields, scal, u, q)
    assert e.value.status == 2


def test_noalloc_rejects_batches_beyond_the_grid_limit():
    """One row of CTAs per instance: more than 65535 instances is refused
    with UNSUPPORTED before any launch, even when B * N fits the scratch."""
    from paper_2502_18377_b300.binding import MpnError, apply_reduced_noalloc, make_desc
    geom = dict(n=(3, 3), step=(0.5, 0.5), periodic=(False, False))
    B = 70000
    desc = make_desc(geom, B, [-1] * 5, 0)
    u = torch.zeros((B, 9), device="cuda")
    q = torch.zeros((B, 9), device="cuda")
    scal = torch.zeros((5, B), device="cuda")
    with pytest.raises(MpnError) as e:
        apply_reduced_noalloc(desc, None, scal, u, q)
    assert e.value.status == 2
