"""Learned warm start: a 4-layer 3x3x3 convolutional network that predicts u
from the coefficient fields and the right-hand side of a PDE instance.

Inference and training run in the library's kernels (BF16 tensor-core
convolutions with FP32 accumulation, FP32-accumulated weight gradients, Adam
on FP32 master weights); this module only holds the parameters and calls the
C ABI layer by layer.  The prediction is handed to the solver as u0; the
solver still iterates to the same tolerance, so the network can only change
how many iterations that takes, never the answer.

Layers (padded channels): (F+2 -> 16) -> 32 ReLU -> 32 ReLU -> 32 ReLU -> 16
(channel 0 is u / out_scale).  Inputs: the coefficient fields, the right-hand
side and its running sum over the time planes (the solution depends on the
forcing of every earlier plane, beyond the layers' 9-plane reach).  Activations are channels-last BF16 [B][N][C].
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from .binding import MpnConvDesc, MpnError, _check_numel, _ptr, _stream, load

LAYERS = [(16, 32), (32, 32), (32, 32), (32, 16)]
RELU, F32, BIAS = 1, 2, 4


def _chk(s, where):
    if s != 0:
        raise MpnError(s, where)


def allreduce_mean(tensors, group=None):
    """Averages `tensors` in place over the ranks of the process group, in one
    all-reduce of a flat buffer (sum, then division by the world size): with
    an equal batch shard per rank, the mean of the per-rank gradients of the
    per-rank mean loss is the gradient of the full-batch mean loss.  NCCL for
    GPU tensors, gloo for CPU tensors; a no-op without a multi-rank group.
    Raises if a rank has left (the collective fails or times out), so a
    failed rank is reported, never waited on forever."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return
    flat = torch.cat([t.reshape(-1) for t in tensors])
    dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
    flat /= dist.get_world_size(group)
    off = 0
    for t in tensors:
        n = t.numel()
        t.copy_(flat[off:off + n].view_as(t))
        off += n


class WarmStartNet:
    def __init__(self, geom: dict, batch: int, nfields: int, seed: int = 0, lr: float = 1e-3,
                 device="cuda"):
        n = tuple(geom["n"])
        if len(n) != 3:
            raise ValueError("the warm-start network works on (t, x, y) grids")
        if nfields + 2 > 16:
            raise ValueError("at most 14 coefficient fields")
        self.lib = load()
        self.geom, self.B, self.F, self.N = geom, batch, nfields, int(np.prod(n))
        self.dev = torch.device(device)
        self.lr, self.b1, self.b2, self.eps, self.step = lr, 0.9, 0.999, 1e-8, 0
        self.desc = []
        for ci, co in LAYERS:
            d = MpnConvDesc()
            for k in range(3):
                d.n[k] = n[k]
                d.periodic[k] = int(geom["periodic"][k])
            d.batch, d.cin, d.cout = batch, ci, co
            self.desc.append(d)
        rng = np.random.default_rng(seed)
        self.w, self.wb, self.b, self.m, self.v = [], [], [], [], []
        real_in = [nfields + 2, 32, 32, 32]
        real_out = [32, 32, 32, 1]
        for (ci, co), ri, ro in zip(LAYERS, real_in, real_out):
            w = np.zeros((27, co, ci), dtype=np.float32)
            w[:, :ro, :ri] = rng.normal(scale=np.sqrt(2.0 / (27 * ri)), size=(27, ro, ri))
            if ro == 1:
                w *= 0.1
            wt = torch.tensor(w, device=self.dev)
            self.w.append(wt)
            self.wb.append(wt.to(torch.bfloat16).contiguous())
            self.b.append(torch.zeros(co, device=self.dev))
        self.m = [torch.zeros_like(t) for t in self.w] + [torch.zeros_like(t) for t in self.b]
        self.v = [torch.zeros_like(t) for t in self.w] + [torch.zeros_like(t) for t in self.b]
        self.in_scale = torch.ones(16, device=self.dev)
        self.out_scale = 1.0
        self._ws = None

    # ------------------------------------------------------------ scaling
    def fit_scales(self, fields, rhs, u):
        """Per-channel input scales and the output scale from training data
        (inverse RMS), so that the network sees O(1) values."""
        sc = np.ones(16, dtype=np.float32)
        for f in range(self.F):
            sc[f] = 1.0 / max(float(fields[f].float().pow(2).mean().sqrt()), 1e-12)
        sc[self.F] = 1.0 / max(float(rhs.float().pow(2).mean().sqrt()), 1e-12)
        nt = int(self.geom["n"][0])
        tsum = rhs.float().reshape(rhs.shape[0], nt, -1).cumsum(1)
        sc[self.F + 1] = 1.0 / max(float(tsum.pow(2).mean().sqrt()), 1e-12)
        self.in_scale = torch.tensor(sc, device=self.dev)
        self.out_scale = max(float(u.float().pow(2).mean().sqrt()), 1e-12)

    # ------------------------------------------------------------ inference
    def _workspace(self):
        if self._ws is None:
            B, N = self.B, self.N
            bf = torch.bfloat16
            self._ws = dict(
                x0=torch.empty((B, N, 16), device=self.dev, dtype=bf),
                a=[torch.empty((B, N, 32), device=self.dev, dtype=bf) for _ in range(3)],
                y=torch.empty((B, N, 16), device=self.dev),
                gy=torch.empty((B, N, 16), device=self.dev),
                g16=torch.empty((B, N, 16), device=self.dev, dtype=bf),
                g32=torch.empty((B, N, 32), device=self.dev, dtype=bf),
                dx=torch.empty((B, N, 32), device=self.dev),
                wt=torch.empty(27 * 32 * 32, device=self.dev, dtype=bf),
                loss=torch.empty((B, 64), device=self.dev),
                u0=torch.empty((B, N), device=self.dev),
                dw=[torch.empty_like(t) for t in self.w],
                db=[torch.empty_like(t) for t in self.b],
            )
            nbytes = max(self.lib.mpn_conv3d_wgrad_scratch_bytes(ctypes.byref(d)) for d in self.desc)
            self._ws["scratch"] = torch.empty(nbytes // 4 + 1, device=self.dev)
        return self._ws

    def _forward(self, fields, rhs):
        # the kernels read F*B*N field values and B*N right-hand-side values
        if self.F:
            _check_numel("fields", fields, self.F * self.B * self.N)
        _check_numel("rhs", rhs, self.B * self.N)
        ws = self._workspace()
        L, st = self.lib, _stream()
        _chk(L.mpn_pack_inputs(ctypes.byref(self.desc[0]), self.F, _ptr(fields) if self.F else None, _ptr(rhs),
                               _ptr(self.in_scale), _ptr(ws["x0"]), st), "pack")
        x = ws["x0"]
        for l in range(4):
            out = ws["a"][l] if l < 3 else ws["y"]
            flags = (RELU | BIAS) if l < 3 else (F32 | BIAS)
            _chk(L.mpn_conv3d_forward(ctypes.byref(self.desc[l]), _ptr(x), _ptr(self.wb[l]), _ptr(self.b[l]),
                                      _ptr(out), flags, st), "conv forward")
            x = out
        return ws["y"]

    def predict(self, fields, rhs):
        """u0 [B][N] (FP32) for the solver's warm start."""
        y = self._forward(fields, rhs)
        ws = self._ws
        _chk(self.lib.mpn_unpack_u(ctypes.byref(self.desc[3]), _ptr(y), ctypes.c_float(self.out_scale),
                                   _ptr(ws["u0"]), _stream()), "unpack")
        return ws["u0"]

    # ------------------------------------------------------------ training
    def gradients(self, fields, rhs, u_target):
        """Loss (MSE of u / out_scale) and parameter gradients into the
        workspace (dw, db); returns the loss as a device scalar."""
        ws = self._workspace()
        L, st = self.lib, _stream()
        y = self._forward(fields, rhs)
        _check_numel("u_target", u_target, self.B * self.N)
        tgt = (u_target / self.out_scale).contiguous()
        _chk(L.mpn_mse_u(ctypes.byref(self.desc[3]), _ptr(y), _ptr(tgt), _ptr(ws["gy"]), _ptr(ws["loss"]), st), "mse")
        acts = [ws["x0"]] + ws["a"]
        g = ws["gy"]                       # FP32 gradient w.r.t. the layer output
        for l in (3, 2, 1, 0):
            ci, co = LAYERS[l]
            gb = ws["g16"] if co == 16 else ws["g32"]
            mask = None if l == 3 else acts[l + 1]
            _chk(L.mpn_relu_mask(g.numel(), _ptr(g), _ptr(mask) if mask is not None else None, _ptr(gb), st), "mask")
            _chk(L.mpn_conv3d_backward_weights(ctypes.byref(self.desc[l]), _ptr(gb), _ptr(acts[l]),
                                               _ptr(ws["scratch"]), _ptr(ws["dw"][l]), _ptr(ws["db"][l]), st),
                 "conv backward weights")
            if l > 0:
                _chk(L.mpn_conv3d_backward_data(ctypes.byref(self.desc[l]), _ptr(gb), _ptr(self.wb[l]),
                                                _ptr(ws["wt"]), _ptr(ws["dx"]), st), "conv backward data")
                g = ws["dx"]
        return ws["loss"].sum() / (self.B * self.N)

    def train_step(self, fields, rhs, u_target, group=None):
        """One Adam step on this rank's batch; under a multi-rank process
        group the weight and bias gradients are first averaged over the ranks
        (data parallelism: every rank holds the same parameters)."""
        loss = self.gradients(fields, rhs, u_target)
        ws = self._ws
        allreduce_mean(ws["dw"] + ws["db"], group)
        self.step += 1
        st = _stream()
        params = self.w + self.b
        grads = ws["dw"] + ws["db"]
        copies = self.wb + [None] * 4
        for k, (p, gr, cp) in enumerate(zip(params, grads, copies)):
            _chk(self.lib.mpn_adam_step(p.numel(), _ptr(p), _ptr(gr), _ptr(self.m[k]), _ptr(self.v[k]),
                                        ctypes.c_float(self.lr), ctypes.c_float(self.b1), ctypes.c_float(self.b2),
                                        ctypes.c_float(self.eps), self.step, _ptr(cp) if cp is not None else None, st),
                 "adam")
        return loss

    # ------------------------------------------------------------ checkpoint
    def state_dict(self):
        return dict(w=[t.cpu() for t in self.w], b=[t.cpu() for t in self.b], m=[t.cpu() for t in self.m],
                    v=[t.cpu() for t in self.v], step=self.step, in_scale=self.in_scale.cpu(),
                    out_scale=self.out_scale, lr=self.lr)

    def load_state_dict(self, sd):
        for dst, src in zip(self.w + self.b + self.m + self.v, sd["w"] + sd["b"] + sd["m"] + sd["v"]):
            dst.copy_(src.to(self.dev))
        self.wb = [t.to(torch.bfloat16).contiguous() for t in self.w]
        self.step, self.lr = sd["step"], sd["lr"]
        self.in_scale = sd["in_scale"].to(self.dev)
        self.out_scale = sd["out_scale"]


class WarmStartTrainer:
    """Epochs over a fixed list of training batches (fields, rhs, u) in a
    seeded order: one permutation per epoch from a CPU generator.  Its
    checkpoint holds the network's parameters, Adam moments and step, the
    generator's state and the data cursor (epoch, permutation, position), so
    a run resumed from it repeats the uninterrupted run bit for bit (the
    layer kernels and their reductions are deterministic)."""

    def __init__(self, net: WarmStartNet, batches, seed: int = 0, group=None):
        self.net, self.batches, self.group = net, batches, group
        self.gen = torch.Generator().manual_seed(seed)
        self.epoch, self.pos = 0, 0
        self.perm = torch.randperm(len(batches), generator=self.gen)

    def step(self):
        """One Adam step on the next batch; returns its loss (device scalar)."""
        if self.pos == len(self.perm):
            self.epoch += 1
            self.pos = 0
            self.perm = torch.randperm(len(self.batches), generator=self.gen)
        f, r, u = self.batches[int(self.perm[self.pos])]
        self.pos += 1
        return self.net.train_step(f, r, u, self.group)

    def state_dict(self):
        return dict(net=self.net.state_dict(), gen=self.gen.get_state(), epoch=self.epoch, pos=self.pos,
                    perm=self.perm.clone())

    def load_state_dict(self, sd):
        self.net.load_state_dict(sd["net"])
        self.gen.set_state(sd["gen"])
        self.epoch, self.pos, self.perm = sd["epoch"], sd["pos"], sd["perm"].clone()
