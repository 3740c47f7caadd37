"""Why the point-local recovery of the derivative unknowns (and the gradient
pass built on it) takes its difference forms in FP64: at the benchmark's
finest transport grid (32 x 256 x 256, x and y periodic on [0, 2 pi)) the
second difference u+ - 2u + u- of a smooth field is about 1e-2 of u, so FP32
differences lose about five digits of the u_xx block, while FP64 differences
followed by FP32 arithmetic (scaling by 1/s, 1/s^2 and the products after
the cancellation) stay at FP32 rounding.  Plain arithmetic on a seeded
smooth field (spectrum ~ k^-3), no solver involved."""
import numpy as np


def _field(nt=32, n=256, modes=8, seed=0):
    t = np.linspace(0.0, 1.0, nt)[:, None, None]
    x = (np.arange(n) * 2 * np.pi / n)[None, :, None]
    y = (np.arange(n) * 2 * np.pi / n)[None, None, :]
    rng = np.random.default_rng(seed)
    u = np.zeros((nt, n, n))
    for k in range(1, modes + 1):
        a, b, c = rng.normal(size=3)
        u += k ** -3.0 * a * np.sin(k * x + b) * np.cos(k * y + c) * np.exp(-0.3 * t)
    return u, 2 * np.pi / n


def _z(u, s, diff_dtype, scale_dtype):
    """u and its x derivatives (central first and second difference forms,
    Eq. 5) with the differences and the scaling in the given precisions."""
    v = u.astype(diff_dtype)
    d1 = (np.roll(v, -1, 1) - np.roll(v, 1, 1)) / diff_dtype(2)
    d2 = np.roll(v, -1, 1) - diff_dtype(2) * v + np.roll(v, 1, 1)
    d1, d2 = d1.astype(scale_dtype), d2.astype(scale_dtype)
    ux = (d1 / scale_dtype(s)).astype(np.float64)
    uxx = (d2 / scale_dtype(s * s)).astype(np.float64)
    return np.concatenate([u.ravel(), ux.ravel(), uxx.ravel()])


def test_fp32_differences_miss_the_tolerance_fp64_differences_keep_it():
    u, s = _field()
    ref = _z(u, s, np.float64, np.float64)
    rel = lambda a: np.linalg.norm(a - ref) / np.linalg.norm(ref)
    e32 = rel(_z(u, s, np.float32, np.float32))
    emix = rel(_z(u, s, np.float64, np.float32))
    assert e32 > 1e-6, e32          # measured 1.8e-5: above the 1e-6 bar of the solves
    assert emix < 1e-7, emix        # measured 4.5e-8
