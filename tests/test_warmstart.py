"""Warm-start network: layer kernels against the FP64 CPU oracle, network
gradients against reverse-mode autograd through the oracle network, and what
a trained network gains for the solver.

Both sides get the same BF16-rounded activations and weights.  The library
accumulates in FP32 and rounds stored activations / gradients to BF16
(relative rounding 2^-8 = 3.9e-3), so layer outputs are compared at 1e-2 and
multi-layer gradients at 5e-2 (relative L2).
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import conv as oc
from paper_2502_18377_b300 import workloads as wl

pytestmark = pytest.mark.gpu


def _rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _desc(n, periodic, B, ci, co):
    from paper_2502_18377_b300.binding import MpnConvDesc
    d = MpnConvDesc()
    for k in range(3):
        d.n[k], d.periodic[k] = n[k], int(periodic[k])
    d.batch, d.cin, d.cout = B, ci, co
    return d


def _bf(t):
    return t.to(torch.bfloat16).to(torch.float64)


@pytest.mark.parametrize("ci,co,flags", [(16, 32, 5), (32, 32, 5), (32, 16, 6), (32, 32, 2)])
@pytest.mark.parametrize("periodic", [(False, True, True), (False, False, True)])
def test_conv_forward_matches_oracle(ci, co, flags, periodic):
    from paper_2502_18377_b300.binding import _ptr, _stream, load
    lib = load()
    n, B = (6, 10, 16), 2
    N = int(np.prod(n))
    g = torch.Generator().manual_seed(ci + co + flags)
    x = torch.randn(B, N, ci, generator=g, dtype=torch.float64)
    w = torch.randn(27, co, ci, generator=g, dtype=torch.float64) * 0.1
    b = torch.randn(co, generator=g, dtype=torch.float64)
    xb, wb = _bf(x), _bf(w)
    ref = oc.conv3d(xb, wb, b if flags & 4 else None, n, periodic, relu=bool(flags & 1))
    xd = xb.to(torch.bfloat16).cuda()
    wd = wb.to(torch.bfloat16).cuda()
    bd = b.float().cuda()
    out = torch.empty(B, N, co, device="cuda", dtype=torch.float32 if flags & 2 else torch.bfloat16)
    d = _desc(n, periodic, B, ci, co)
    assert lib.mpn_conv3d_forward(ctypes.byref(d), _ptr(xd), _ptr(wd), _ptr(bd), _ptr(out), flags, _stream()) == 0
    got = out.double().cpu()
    assert _rel(got, ref) <= 1e-2, _rel(got, ref)


MMA_SYNC = 8   # MPN_CONV_MMA_SYNC: the legacy warp-level kernel


@pytest.mark.parametrize("ci,co,flags", [(16, 32, 5), (32, 32, 5), (32, 16, 6), (32, 32, 2), (32, 32, 0)])
@pytest.mark.parametrize("n,B,periodic", [((6, 10, 16), 2, (False, True, True)),     # 960 points: a ragged tile
                                          ((5, 7, 9), 3, (False, False, False)),
                                          ((32, 64, 64), 2, (False, True, True)),   # more tiles than CTAs
                                          # rows of whole 128-point tiles: the row-staged kernel
                                          ((3, 2, 128), 2, (False, True, True)),
                                          ((4, 3, 256), 1, (False, False, False)),
                                          ((16, 32, 128), 2, (False, True, True))])
def test_conv_tcgen05_matches_mma_sync_and_oracle(ci, co, flags, n, B, periodic):
    """The tcgen05 convolution (the default; rows of n_y % 128 == 0 take its
    row-staged kernel) against the mma.sync kernel on the same BF16 inputs (FP32 accumulation in both, summed in different orders:
    1e-5 for FP32 output, one BF16 rounding for BF16 output) and, on the small
    grids, against the oracle."""
    from paper_2502_18377_b300.binding import _ptr, _stream, load
    lib = load()
    N = int(np.prod(n))
    g = torch.Generator().manual_seed(7 * ci + co + flags + N)
    xb = _bf(torch.randn(B, N, ci, generator=g, dtype=torch.float64))
    wb = _bf(torch.randn(27, co, ci, generator=g, dtype=torch.float64) * 0.1)
    b = torch.randn(co, generator=g, dtype=torch.float64)
    xd, wd, bd = xb.to(torch.bfloat16).cuda(), wb.to(torch.bfloat16).cuda(), b.float().cuda()
    dt = torch.float32 if flags & 2 else torch.bfloat16
    d = _desc(n, periodic, B, ci, co)
    outs = []
    for extra in (0, MMA_SYNC, 0):
        out = torch.full((B, N, co), float("nan"), device="cuda", dtype=dt)
        assert lib.mpn_conv3d_forward(ctypes.byref(d), _ptr(xd), _ptr(wd), _ptr(bd), _ptr(out), flags | extra,
                                      _stream()) == 0
        torch.cuda.synchronize()
        outs.append(out.double().cpu())
    tcg, legacy, again = outs
    flag = ctypes.c_int(-1)
    assert lib.mpn_conv_take_error(ctypes.byref(flag)) == 0 and flag.value == 0   # no bounded wait gave up
    assert torch.isfinite(tcg).all()
    assert torch.equal(tcg, again)                       # deterministic
    assert _rel(tcg, legacy) <= (1e-5 if flags & 2 else 8e-3), _rel(tcg, legacy)
    if N <= 1024:
        ref = oc.conv3d(xb, wb, b if flags & 4 else None, n, periodic, relu=bool(flags & 1))
        assert _rel(tcg, ref) <= 1e-2, _rel(tcg, ref)


@pytest.mark.parametrize("co", [32, 16])
def test_conv_backward_matches_oracle(co):
    from paper_2502_18377_b300.binding import _ptr, _stream, load
    lib = load()
    n, B, ci, periodic = (5, 8, 12), 2, 32, (False, True, True)
    N = int(np.prod(n))
    g = torch.Generator().manual_seed(co)
    x = _bf(torch.randn(B, N, ci, generator=g, dtype=torch.float64))
    w = _bf(torch.randn(27, co, ci, generator=g, dtype=torch.float64) * 0.1)
    gy = _bf(torch.randn(B, N, co, generator=g, dtype=torch.float64))
    xr = x.clone().requires_grad_(True)
    wr = w.clone().requires_grad_(True)
    br = torch.zeros(co, dtype=torch.float64, requires_grad=True)
    y = oc.conv3d(xr, wr, br, n, periodic)
    (y * gy).sum().backward()
    d = _desc(n, periodic, B, ci, co)
    gyd = gy.to(torch.bfloat16).cuda()
    wd = w.to(torch.bfloat16).cuda()
    xd = x.to(torch.bfloat16).cuda()
    dx = torch.empty(B, N, ci, device="cuda")
    wt = torch.empty(27 * ci * co, device="cuda", dtype=torch.bfloat16)
    assert lib.mpn_conv3d_backward_data(ctypes.byref(d), _ptr(gyd), _ptr(wd), _ptr(wt), _ptr(dx), _stream()) == 0
    nb = lib.mpn_conv3d_wgrad_scratch_bytes(ctypes.byref(d))
    scratch = torch.empty(nb // 4 + 1, device="cuda")
    dw = torch.empty(27, co, ci, device="cuda")
    db = torch.empty(co, device="cuda")
    assert lib.mpn_conv3d_backward_weights(ctypes.byref(d), _ptr(gyd), _ptr(xd), _ptr(scratch), _ptr(dw), _ptr(db),
                                           _stream()) == 0
    torch.cuda.synchronize()
    assert _rel(dx.cpu(), xr.grad) <= 1e-5
    assert _rel(dw.cpu(), wr.grad) <= 1e-5
    assert _rel(db.cpu(), br.grad) <= 1e-5


def _small_family(batch, seed_base):
    return wl.reaction_diffusion_2d(batch=batch, n=(8, 16, 16), seed_base=seed_base)


def test_network_gradients_match_oracle():
    from paper_2502_18377_b300.warmstart import WarmStartNet
    w = _small_family(2, 9000)
    dev = lambda a: torch.tensor(np.asarray(a, dtype=np.float32), device="cuda")
    net = WarmStartNet(w.geom, w.batch, 2, seed=3)
    fields, rhs = dev(w.fields), dev(w.rhs)
    u = dev(w.target)                  # any target works for a gradient check
    net.fit_scales(fields, rhs, u)
    loss = net.gradients(fields, rhs, u)
    torch.cuda.synchronize()
    ws = net._ws
    # oracle: same BF16 packed inputs and weights, FP64 everywhere else
    x0 = ws["x0"].double().cpu()
    wts = [_bf(t.double().cpu()).requires_grad_(True) for t in net.w]
    bs = [t.double().cpu().requires_grad_(True) for t in net.b]
    y = oc.net_forward(x0, wts, bs, w.geom["n"], w.geom["periodic"])
    tgt = (u / net.out_scale).double().cpu()
    lref = ((y[:, :, 0] - tgt) ** 2).mean()
    lref.backward()
    assert abs(float(loss) - float(lref)) <= 5e-2 * float(lref)
    for l in range(4):
        assert _rel(ws["dw"][l].cpu(), wts[l].grad) <= 5e-2, (l, _rel(ws["dw"][l].cpu(), wts[l].grad))
        assert _rel(ws["db"][l].cpu(), bs[l].grad) <= 5e-2, (l, _rel(ws["db"][l].cpu(), bs[l].grad))


def test_trained_network_gains():
    """Train on solves of the plain method, then on held-out instances the
    prediction beats a zero start and the warm-started solve needs no more
    PCG iterations than the cold one, reaching the same solution."""
    from paper_2502_18377_b300.binding import Solver
    from paper_2502_18377_b300.warmstart import WarmStartNet
    dev = lambda a: torch.tensor(np.asarray(a, dtype=np.float32), device="cuda")
    B = 4
    train = []
    for k in range(6):
        w = _small_family(B, 10000 + 10 * k)
        s = Solver(w.geom, B, w.field_of, 2)
        args = (dev(w.fields), dev(w.scalars), dev(w.rhs), dev(w.omega))
        z = s.forward(*args)
        train.append((args[0], args[2], z[:, 0].contiguous()))
    net = WarmStartNet(w.geom, B, 2, seed=0, lr=2e-3)
    net.fit_scales(*train[0])
    for it in range(150):
        f, r, u = train[it % len(train)]
        net.train_step(f, r, u)
    test = _small_family(B, 20000)
    s = Solver(test.geom, B, test.field_of, 2)
    args = (dev(test.fields), dev(test.scalars), dev(test.rhs), dev(test.omega))
    z_cold = s.forward(*args)
    cold = dict(s.last_stats)
    u0 = net.predict(args[0], args[2]).clone()
    u = z_cold[:, 0]
    err0 = float((u0 - u).norm() / u.norm())
    assert err0 < 1.0, err0
    z_warm = s.forward(*args, u0=u0)
    warm = dict(s.last_stats)
    print("warm-start gain:", dict(err0=err0, cold=cold, warm=warm))
    assert warm["pcg_iters"] <= cold["pcg_iters"], (warm, cold)
    assert float((z_warm - z_cold).norm() / z_cold.norm()) <= 2e-6


def test_trainer_checkpoint_resume_is_bitwise():
    """Train 5 steps, checkpoint (parameters, Adam moments, step, scales,
    generator state, data cursor), resume in a fresh trainer for 6 more
    steps: every parameter and moment equals that of an uninterrupted
    11-step run bit for bit (the cursor crosses an epoch boundary)."""
    import io
    from paper_2502_18377_b300.warmstart import WarmStartNet, WarmStartTrainer
    dev = lambda a: torch.tensor(np.asarray(a, dtype=np.float32), device="cuda")
    batches = []
    for k in range(4):
        w = _small_family(2, 30000 + 10 * k)
        batches.append((dev(w.fields), dev(w.rhs), dev(w.target)))

    def make():
        net = WarmStartNet(w.geom, 2, 2, seed=5, lr=2e-3)
        net.fit_scales(*batches[0])
        return WarmStartTrainer(net, batches, seed=11)

    full = make()
    for _ in range(11):
        full.step()
    first = make()
    for _ in range(5):
        first.step()
    buf = io.BytesIO()
    torch.save(first.state_dict(), buf)
    buf.seek(0)
    resumed = make()
    resumed.load_state_dict(torch.load(buf))
    for _ in range(6):
        resumed.step()
    torch.cuda.synchronize()
    assert resumed.epoch == full.epoch == 2 and resumed.pos == full.pos
    a, b = full.net, resumed.net
    for x, y in zip(a.w + a.b + a.m + a.v + a.wb, b.w + b.b + b.m + b.v + b.wb):
        assert torch.equal(x, y)
    assert a.step == b.step == 11


def test_packed_inputs():
    """Input channels of the network: the fields and the right-hand side
    scaled, and the running sum over time planes of the right-hand side
    (plain numpy cumulative sum), BF16-rounded; zero padding above."""
    from paper_2502_18377_b300.binding import _ptr, _stream, load
    lib = load()
    w = _small_family(2, 9100)
    n, B, F = w.geom["n"], 2, 2
    d = _desc(n, w.geom["periodic"], B, 16, 32)
    scale = np.array([0.5, 2.0, 3.0, 0.25] + [1.0] * 12, dtype=np.float32)
    fields = torch.tensor(np.asarray(w.fields, dtype=np.float32), device="cuda")
    rhs = torch.tensor(np.asarray(w.rhs, dtype=np.float32), device="cuda")
    x0 = torch.empty((B, w.npoints, 16), device="cuda", dtype=torch.bfloat16)
    sc = torch.tensor(scale, device="cuda")
    assert lib.mpn_pack_inputs(ctypes.byref(d), F, _ptr(fields), _ptr(rhs), _ptr(sc), _ptr(x0), _stream()) == 0
    got = x0.float().cpu().numpy().astype(np.float64)
    f32 = np.asarray(w.fields, dtype=np.float32).astype(np.float64)
    r32 = np.asarray(w.rhs, dtype=np.float32).astype(np.float64)
    tsum = np.cumsum(r32.reshape(B, n[0], -1), axis=1).reshape(B, -1)
    refs = [f32[0] * 0.5, f32[1] * 2.0, r32 * 3.0, tsum * 0.25]
    for c, ref in enumerate(refs):
        assert _rel(got[:, :, c], ref) <= 8e-3, (c, _rel(got[:, :, c], ref))
    assert not np.any(got[:, :, 4:])
