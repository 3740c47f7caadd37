"""Pins of the convolution oracle (warm-start network layers)."""
import numpy as np
import pytest
import torch

from oracle import conv as oc


@pytest.mark.parametrize("periodic", [(False, True, True), (False, False, True), (False, False, False)])
def test_conv_matches_bruteforce(periodic):
    g = torch.Generator().manual_seed(0)
    n = (3, 4, 5)
    x = torch.randn(2, 60, 3, generator=g, dtype=torch.float64)
    w = torch.randn(27, 4, 3, generator=g, dtype=torch.float64)
    b = torch.randn(4, generator=g, dtype=torch.float64)
    ref = oc.conv3d_bruteforce(x, w, b, n, periodic)
    got = oc.conv3d(x, w, b, n, periodic)
    assert torch.allclose(got, ref, atol=1e-12)


def test_conv_identity_and_shift():
    """The centre tap alone copies the input; a single off-centre tap shifts it
    (with wrap in periodic dims, zeros past the time edges)."""
    n = (4, 5, 6)
    x = torch.randn(1, 120, 2, dtype=torch.float64)
    w = torch.zeros(27, 2, 2, dtype=torch.float64)
    w[13] = torch.eye(2, dtype=torch.float64)
    assert torch.allclose(oc.conv3d(x, w, None, n, (False, True, True)), x)
    w = torch.zeros(27, 2, 2, dtype=torch.float64)
    w[14] = torch.eye(2, dtype=torch.float64)          # offset (0, 0, +1): y[p] = x[p + e_y]
    y = oc.conv3d(x, w, None, n, (False, True, True)).reshape(4, 5, 6, 2)
    xs = x.reshape(4, 5, 6, 2)
    assert torch.allclose(y, torch.roll(xs, -1, dims=2))
    w = torch.zeros(27, 2, 2, dtype=torch.float64)
    w[22] = torch.eye(2, dtype=torch.float64)          # offset (+1, 0, 0): time, zero at the last step
    y = oc.conv3d(x, w, None, n, (False, True, True)).reshape(4, 5, 6, 2)
    assert torch.allclose(y[:-1], xs[1:]) and torch.all(y[-1] == 0)
