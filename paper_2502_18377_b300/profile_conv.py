"""Runs one layer of the warm-start network's convolution for profilers (ncu)
and quick timings: the tcgen05 kernel, then (with --both) the mma.sync
kernel on the same inputs.

python -m paper_2502_18377_b300.profile_conv [--batch B] [--grid T X Y]
    [--cin 32] [--cout 32] [--reps K] [--both]
"""
from __future__ import annotations

import argparse
import ctypes
import json

import torch

from .binding import MpnConvDesc, _ptr, _stream, load

MMA_SYNC = 8       # MPN_CONV_MMA_SYNC
RELU_BIAS = 1 | 4  # MPN_CONV_RELU | MPN_CONV_BIAS


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--batch", type=int, default=2)
    ap.add_argument("--grid", type=int, nargs=3, default=(64, 128, 128))
    ap.add_argument("--cin", type=int, default=32)
    ap.add_argument("--cout", type=int, default=32)
    ap.add_argument("--reps", type=int, default=1)
    ap.add_argument("--both", action="store_true", help="also run the mma.sync kernel")
    a = ap.parse_args()
    lib = load()
    n, B, ci, co = tuple(a.grid), a.batch, a.cin, a.cout
    N = n[0] * n[1] * n[2]
    d = MpnConvDesc()
    for k in range(3):
        d.n[k], d.periodic[k] = n[k], int(k > 0)
    d.batch, d.cin, d.cout = B, ci, co
    g = torch.Generator(device="cuda").manual_seed(1)
    x = torch.randn(B, N, ci, device="cuda", generator=g).to(torch.bfloat16)
    w = (0.1 * torch.randn(27, co, ci, device="cuda", generator=g)).to(torch.bfloat16)
    b = torch.randn(co, device="cuda", generator=g)
    out = torch.empty(B, N, co, device="cuda", dtype=torch.bfloat16)
    res = {}
    for name, extra in (("tcgen05", 0), ("mma_sync", MMA_SYNC))[: 2 if a.both else 1]:
        if a.reps > 1:   # one untimed launch (first-call set-up, caches)
            lib.mpn_conv3d_forward(ctypes.byref(d), _ptr(x), _ptr(w), _ptr(b), _ptr(out), RELU_BIAS | extra, _stream())
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(a.reps):
            s = lib.mpn_conv3d_forward(ctypes.byref(d), _ptr(x), _ptr(w), _ptr(b), _ptr(out), RELU_BIAS | extra,
                                       _stream())
            if s != 0:
                raise RuntimeError(f"mpn_conv3d_forward: status {s}")
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / a.reps
        res[name] = {"ms": ms, "TFLOP/s": 2 * 27 * ci * co * B * N / ms / 1e9}
    print(json.dumps({"batch": B, "grid": list(n), "cin": ci, "cout": co, **res}))


if __name__ == "__main__":
    main()
