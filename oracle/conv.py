"""FP64 CPU reference of the warm-start network's layer operations.

TEST INFRASTRUCTURE ONLY (see the package docstring).  The paper has no such
network; this is the plain definition of a 3x3x3 convolution on the
(t, x, y) grid with zero padding in t and periodic (or zero) padding in x, y:
    y[b, p, co] = bias[co] + sum_{tap, ci} W[tap, co, ci] x[b, p + off(tap), ci],
    off(tap) = (tap // 9 - 1, (tap // 3) % 3 - 1, tap % 3 - 1),
evaluated with torch's CPU conv3d after explicit padding, and its gradients
by reverse-mode autograd.  Layouts match the library: x [B][N][C]
channels-last, W [27][Cout][Cin].
"""
from __future__ import annotations

import torch
import torch.nn.functional as F


def _to_ncdhw(x, n):
    B, N, C = x.shape
    return x.reshape(B, n[0], n[1], n[2], C).permute(0, 4, 1, 2, 3)


def conv3d(x, w, bias, n, periodic, relu=False):
    """x [B][N][Cin], w [27][Cout][Cin], bias [Cout] or None -> [B][N][Cout]."""
    x5 = _to_ncdhw(x, n)
    if periodic[2]:
        x5 = torch.cat([x5[..., -1:], x5, x5[..., :1]], dim=4)
    else:
        x5 = F.pad(x5, (1, 1, 0, 0, 0, 0))
    if periodic[1]:
        x5 = torch.cat([x5[:, :, :, -1:], x5, x5[:, :, :, :1]], dim=3)
    else:
        x5 = F.pad(x5, (0, 0, 1, 1, 0, 0))
    x5 = F.pad(x5, (0, 0, 0, 0, 1, 1))                       # time: zero padding
    k = w.reshape(3, 3, 3, w.shape[1], w.shape[2]).permute(3, 4, 0, 1, 2)
    y = F.conv3d(x5, k, bias)
    if relu:
        y = torch.relu(y)
    B, C = y.shape[0], y.shape[1]
    return y.permute(0, 2, 3, 4, 1).reshape(B, -1, C)


def conv3d_bruteforce(x, w, bias, n, periodic):
    """The defining sum with explicit loops (tiny grids only)."""
    B, N, Ci = x.shape
    Co = w.shape[1]
    y = torch.zeros(B, N, Co, dtype=x.dtype)
    for b in range(B):
        for t in range(n[0]):
            for i in range(n[1]):
                for j in range(n[2]):
                    p = (t * n[1] + i) * n[2] + j
                    acc = bias.clone() if bias is not None else torch.zeros(Co, dtype=x.dtype)
                    for tap in range(27):
                        dt, di, dj = tap // 9 - 1, (tap // 3) % 3 - 1, tap % 3 - 1
                        tt, ii, jj = t + dt, i + di, j + dj
                        if tt < 0 or tt >= n[0]:
                            continue
                        if not 0 <= ii < n[1]:
                            if not periodic[1]:
                                continue
                            ii %= n[1]
                        if not 0 <= jj < n[2]:
                            if not periodic[2]:
                                continue
                            jj %= n[2]
                        q = (tt * n[1] + ii) * n[2] + jj
                        acc = acc + w[tap] @ x[b, q]
                    y[b, p] = acc
    return y


def net_forward(x0, ws, bs, n, periodic):
    """The 4-layer network: ReLU after layers 1-3, linear output."""
    a = x0
    for l, (w, b) in enumerate(zip(ws, bs)):
        a = conv3d(a, w, b, n, periodic, relu=l < len(ws) - 1)
    return a
