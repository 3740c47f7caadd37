"""ctypes binding of libmpn.so (argument marshalling only).

Every entry point here forwards to the C ABI declared in include/mpn.h; all
arithmetic of the solve runs in the library's CUDA kernels.  PyTorch provides
the device memory and the current stream.  The library must have been built
(``paper_2502_18377_b300.csrc.build.build()``); there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmpn.so")
DEBUG_LIB_PATH = os.path.join(_HERE, "libmpn_debug.so")   # bounds-checked build (MPN_DEBUG)

MPN_REUSE_SETUP = 1
STATUS = {0: "ok", 1: "invalid argument", 2: "unsupported", 3: "not converged",
          4: "non-finite", 5: "diverged", 6: "CUDA error", 7: "out of memory"}


class MpnDesc(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n", ctypes.c_int * 3), ("step", ctypes.c_double * 3),
                ("periodic", ctypes.c_int * 3), ("stencil", ctypes.c_int),
                ("final_time_rows", ctypes.c_int), ("batch", ctypes.c_int),
                ("nfields", ctypes.c_int), ("field_of", ctypes.c_int * 7), ("tol", ctypes.c_double),
                ("max_refine", ctypes.c_int), ("inner_iters", ctypes.c_int),
                ("cheb_degree", ctypes.c_int), ("coarse_min", ctypes.c_int),
                ("max_coarse", ctypes.c_int), ("fused_coarse", ctypes.c_int),
                ("fused_step", ctypes.c_int), ("krylov", ctypes.c_int), ("coarsen_time", ctypes.c_int),
                ("direct", ctypes.c_int), ("variable_steps", ctypes.c_int),
                ("bc_alpha", ctypes.c_double * 3), ("bc_beta", ctypes.c_double * 3),
                ("adj_inner_iters", ctypes.c_int)]

KRYLOV = {"cg": 0, "fgmres": 1}


class MpnConvDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("periodic", ctypes.c_int * 3), ("batch", ctypes.c_int),
                ("cin", ctypes.c_int), ("cout", ctypes.c_int)]


class MpnStats(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int), ("pcg_iters", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("rel_update", ctypes.c_double),
                ("pred_error", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = ctypes.c_void_p
EXPORTS = {
    "mpn_default_desc": (ctypes.c_int, [ctypes.POINTER(MpnDesc)]),
    "mpn_create": (ctypes.c_int, [ctypes.POINTER(MpnDesc), ctypes.POINTER(_P)]),
    "mpn_workspace_bytes": (ctypes.c_size_t, [_P]),
    "mpn_levels": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "mpn_fused_level": (ctypes.c_int, [_P]),
    "mpn_forward": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, ctypes.POINTER(MpnStats), _P]),
    "mpn_adjoint": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, ctypes.c_int,
                                   ctypes.POINTER(MpnStats), _P]),
    "mpn_generation": (ctypes.c_longlong, [_P]),
    "mpn_set_steps": (ctypes.c_int, [_P, _P, _P]),
    "mpn_step_grads": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "mpn_inject_wait_failure": (ctypes.c_int, [_P]),
    "mpn_mse_grad": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "mpn_debug_take": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    "mpn_apply_reduced": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "mpn_profile": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_longlong)]),
    "mpn_apply_reduced_noalloc": (ctypes.c_int, [ctypes.POINTER(MpnDesc), _P, _P, _P, _P, _P]),
    "mpn_conv3d_forward": (ctypes.c_int, [ctypes.POINTER(MpnConvDesc), _P, _P, _P, _P, ctypes.c_int, _P]),
    "mpn_conv_take_error": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int)]),
    "mpn_conv3d_backward_data": (ctypes.c_int, [ctypes.POINTER(MpnConvDesc), _P, _P, _P, _P, _P]),
    "mpn_conv3d_wgrad_scratch_bytes": (ctypes.c_size_t, [ctypes.POINTER(MpnConvDesc)]),
    "mpn_conv3d_backward_weights": (ctypes.c_int, [ctypes.POINTER(MpnConvDesc), _P, _P, _P, _P, _P, _P]),
    "mpn_relu_mask": (ctypes.c_int, [ctypes.c_longlong, _P, _P, _P, _P]),
    "mpn_adam_step": (ctypes.c_int, [ctypes.c_longlong, _P, _P, _P, _P, ctypes.c_float, ctypes.c_float,
                                     ctypes.c_float, ctypes.c_float, ctypes.c_int, _P, _P]),
    "mpn_pack_inputs": (ctypes.c_int, [ctypes.POINTER(MpnConvDesc), ctypes.c_int, _P, _P, _P, _P, _P]),
    "mpn_mse_u": (ctypes.c_int, [ctypes.POINTER(MpnConvDesc), _P, _P, _P, _P, _P]),
    "mpn_unpack_u": (ctypes.c_int, [ctypes.POINTER(MpnConvDesc), _P, ctypes.c_float, _P, _P]),
    "mpn_destroy": (None, [_P]),
    "mpn_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "mpn_last_cuda_error": (ctypes.c_char_p, []),
}

_lib = None


def load(path: str = LIB_PATH):
    """Loads libmpn.so and declares its signatures.  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libmpn.so not built at {path}: run paper_2502_18377_b300.csrc.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class MpnError(RuntimeError):
    def __init__(self, status, where):
        lib = load()
        msg = lib.mpn_strerror(status).decode()
        if status == 6:
            msg += ": " + lib.mpn_last_cuda_error().decode()
        super().__init__(f"{where}: {msg} (status {status})")
        self.status = status


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("tensor must be on a CUDA device")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _check_f32(name, t, shape):
    if t.dtype != torch.float32:
        raise ValueError(f"{name} must be float32")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")


NOALLOC_MAX_POINTS = 4194304


def make_desc(geom: dict, batch: int, field_of, nfields: int) -> MpnDesc:
    """Descriptor for a grid / batch / coefficient layout (solver defaults)."""
    lib = load()
    d = MpnDesc()
    lib.mpn_default_desc(ctypes.byref(d))
    n = tuple(geom["n"])
    D = len(n)
    d.ndim = D
    for k in range(3):
        d.n[k] = n[k] if k < D else 1
        d.step[k] = geom["step"][k] if k < D else 1.0
        d.periodic[k] = int(geom["periodic"][k]) if k < D else 0
    d.stencil = int(geom.get("stencil", 3))
    d.final_time_rows = int(geom.get("final_time_rows", False))
    d.batch = batch
    d.nfields = nfields
    for v in range(7):
        d.field_of[v] = field_of[v] if v < len(field_of) else -1
    return d


def _check_numel(name, t, n, dtype=torch.float32):
    """`dtype` with exactly n elements (the C ABI reads and writes n of them)."""
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if t.numel() != n:
        raise ValueError(f"{name} has {t.numel()} elements, expected {n}")


def apply_reduced_noalloc(desc: MpnDesc, fields, scalars, u, q):
    """q = S u through the allocation-free entry point (q preallocated).

    The descriptor is built apart from the tensors, so their sizes are checked
    against it here: a short q or u would otherwise be read or written out of
    bounds by the kernels."""
    N = 1
    for k in range(desc.ndim):
        N *= desc.n[k]
    B, V = desc.batch, 1 + 2 * desc.ndim
    _check_numel("u", u, B * N)
    _check_numel("q", q, B * N)
    _check_numel("scalars", scalars, V * B)
    if desc.nfields:
        _check_numel("fields", fields, desc.nfields * B * N)
    lib = load()
    s = lib.mpn_apply_reduced_noalloc(ctypes.byref(desc), _ptr(fields) if desc.nfields else None, _ptr(scalars),
                                      _ptr(u), _ptr(q), _stream())
    if s != 0:
        raise MpnError(s, "mpn_apply_reduced_noalloc")
    return q


class Solver:
    """One problem object (grid, batch, coefficient layout) of the C ABI."""

    def __init__(self, geom: dict, batch: int, field_of, nfields: int, tol=1e-7, max_refine=12,
                 inner_iters=5, cheb_degree=5, coarse_min=4, max_coarse=2048, fused_coarse=True,
                 fused_step=3, krylov="cg", coarsen_time=False, direct=False, variable_steps=False,
                 adj_inner_iters=0):
        lib = load()
        d = MpnDesc()
        lib.mpn_default_desc(ctypes.byref(d))
        n = tuple(geom["n"])
        D = len(n)
        d.ndim = D
        for k in range(3):
            d.n[k] = n[k] if k < D else 1
            d.step[k] = geom["step"][k] if k < D else 1.0
            d.periodic[k] = int(geom["periodic"][k]) if k < D else 0
        d.stencil = int(geom.get("stencil", 3))
        d.final_time_rows = int(geom.get("final_time_rows", False))
        d.batch = batch
        d.nfields = nfields
        for v in range(7):
            d.field_of[v] = field_of[v] if v < len(field_of) else -1
        d.tol, d.max_refine, d.inner_iters = tol, max_refine, inner_iters
        d.cheb_degree, d.coarse_min, d.max_coarse = cheb_degree, coarse_min, max_coarse
        d.fused_coarse = int(bool(fused_coarse))
        d.fused_step = int(fused_step)
        d.krylov = KRYLOV[krylov]
        d.coarsen_time = int(bool(coarsen_time))
        d.direct = int(bool(direct))
        d.variable_steps = int(bool(variable_steps))
        d.adj_inner_iters = int(adj_inner_iters)
        # boundary rows alpha u + beta du/dx_d = omega per spatial axis
        # (geom["bc"] = {d: (alpha, beta)}; Dirichlet where absent)
        for k, (a, b) in dict(geom.get("bc", {})).items():
            if not 1 <= int(k) < D:
                raise ValueError(f"boundary kind for axis {k}: only spatial axes 1..{D - 1}")
            d.bc_alpha[int(k)], d.bc_beta[int(k)] = float(a), float(b)
        h = ctypes.c_void_p()
        s = lib.mpn_create(ctypes.byref(d), ctypes.byref(h))
        if s != 0:
            raise MpnError(s, "mpn_create")
        self._h = h
        self.lib = lib
        self.geom = geom
        self.D, self.V, self.B, self.F = D, 1 + 2 * D, batch, nfields
        self.N = 1
        for k in n:
            self.N *= k
        self.field_of = list(field_of)
        self.last_stats = None
        self.variable_steps = bool(variable_steps)
        # intervals per axis: n - 1 on an open axis, n on a periodic one
        self.step_counts = [n[k] if d.periodic[k] else n[k] - 1 for k in range(D)]

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self.lib.mpn_destroy(h)
            self._h = None

    @property
    def workspace_bytes(self):
        return int(self.lib.mpn_workspace_bytes(self._h))

    def debug_take(self):
        """Bounds-checked build: the code of the first out-of-range index a
        kernel formed since the last call (0: none), cleared; None with the
        release library."""
        code = ctypes.c_int()
        s = self.lib.mpn_debug_take(self._h, ctypes.byref(code))
        if s == 2:
            return None
        if s != 0:
            raise MpnError(s, "mpn_debug_take")
        return code.value

    def generation(self):
        """Forward solves completed on this problem so far."""
        return int(self.lib.mpn_generation(self._h))

    def inject_wait_failure(self):
        """Test hook: the next solve reports a kernel's bounded wait giving up
        (MPN_ERR_CUDA) through the device error word, without any fault."""
        s = self.lib.mpn_inject_wait_failure(self._h)
        if s != 0:
            raise MpnError(s, "mpn_inject_wait_failure")

    def fused_level(self):
        """First level of the fused coarse end of the V-cycle, or -1."""
        return int(self.lib.mpn_fused_level(self._h))

    def levels(self):
        nl = ctypes.c_int()
        shapes = (ctypes.c_int * 48)()
        self.lib.mpn_levels(self._h, ctypes.byref(nl), shapes)
        return [tuple(shapes[3 * k + d] for d in range(3)) for k in range(nl.value)]

    def _inputs(self, fields, scalars, rhs, omega):
        _check_f32("scalars", scalars, (self.V, self.B))
        _check_f32("rhs", rhs, (self.B, self.N))
        _check_f32("omega", omega, (self.B, self.N))
        if self.F > 0:
            _check_f32("fields", fields, (self.F, self.B, self.N))

    def forward(self, fields, scalars, rhs, omega, u0=None, z=None, z64=None, allow_not_converged=False):
        """Returns z [B][V][N] (float32); z64 (float64) is filled if given."""
        self._inputs(fields, scalars, rhs, omega)
        BN, BVN = self.B * self.N, self.B * self.V * self.N
        if u0 is not None:
            _check_numel("u0", u0, BN)
        if z is not None:
            _check_numel("z", z, BVN)
        if z64 is not None:
            _check_numel("z64", z64, BVN, torch.float64)
        if z is None:
            z = torch.empty((self.B, self.V, self.N), device=rhs.device, dtype=torch.float32)
        st = MpnStats()
        s = self.lib.mpn_forward(self._h, _ptr(fields) if self.F else None, _ptr(scalars), _ptr(rhs),
                                 _ptr(omega), _ptr(u0), _ptr(z), _ptr(z64), ctypes.byref(st), _stream())
        self.last_stats = st.as_dict()
        if s != 0 and not (s == 3 and allow_not_converged):
            raise MpnError(s, "mpn_forward")
        return z

    def adjoint(self, fields, scalars, rhs, omega, z, g_z, reuse_setup=False, want_dz=False, dz64=None):
        """Returns (dfields, dscalars, drhs, domega[, dz]); dz64 (float64
        [B][V][N]), if given, receives d_z as the FP64 refinement holds it."""
        self._inputs(fields, scalars, rhs, omega)
        _check_f32("g_z", g_z, (self.B, self.V, self.N))
        if z is not None:
            _check_numel("z", z, self.B * self.V * self.N)
        dev = rhs.device
        dfields = torch.empty((max(self.F, 1), self.B, self.N), device=dev, dtype=torch.float32)
        dscal = torch.empty((self.V, self.B), device=dev, dtype=torch.float32)
        drhs = torch.empty((self.B, self.N), device=dev, dtype=torch.float32)
        dom = torch.empty((self.B, self.N), device=dev, dtype=torch.float32)
        dz = torch.empty((self.B, self.V, self.N), device=dev, dtype=torch.float32) if want_dz else None
        if dz64 is not None and (dz64.dtype != torch.float64 or tuple(dz64.shape) != (self.B, self.V, self.N)):
            raise ValueError("dz64 must be float64 [B][V][N]")
        st = MpnStats()
        s = self.lib.mpn_adjoint(self._h, _ptr(fields) if self.F else None, _ptr(scalars), _ptr(rhs),
                                 _ptr(omega), _ptr(z), _ptr(g_z), _ptr(dfields), _ptr(dscal), _ptr(drhs),
                                 _ptr(dom), _ptr(dz), _ptr(dz64), MPN_REUSE_SETUP if reuse_setup else 0,
                                 ctypes.byref(st), _stream())
        self.last_stats = st.as_dict()
        if s != 0:
            raise MpnError(s, "mpn_adjoint")
        out = (dfields[: self.F], dscal, drhs, dom)
        return out + (dz,) if want_dz else out

    def set_steps(self, steps):
        """Per-interval steps of a variable_steps problem: one float32 tensor
        [B, m_d] per axis (time first; m_d = n_d - 1, or n_d on a periodic
        axis).  The library copies them; the next solves use them."""
        if not self.variable_steps:
            raise ValueError("set_steps needs a variable_steps problem")
        if len(steps) != self.D:
            raise ValueError(f"expected {self.D} step tensors")
        for k, (t, m) in enumerate(zip(steps, self.step_counts)):
            _check_f32(f"steps[{k}]", t, (self.B, m))
        flat = torch.cat([t.reshape(-1) for t in steps]).contiguous()
        s = self.lib.mpn_set_steps(self._h, _ptr(flat), _stream())
        if s != 0:
            raise MpnError(s, "mpn_set_steps")

    def step_grads(self, z64, dz64):
        """dl/dsteps (one float32 tensor [B, m_d] per axis) from the FP64
        forward solution and the FP64 adjoint solution ([B][V][N] each)."""
        for name, t in (("z64", z64), ("dz64", dz64)):
            if t.dtype != torch.float64 or tuple(t.shape) != (self.B, self.V, self.N):
                raise ValueError(f"{name} must be float64 [B][V][N]")
        out = torch.empty(self.B * sum(self.step_counts), device=z64.device, dtype=torch.float32)
        s = self.lib.mpn_step_grads(self._h, _ptr(z64), _ptr(dz64), _ptr(out), _stream())
        if s != 0:
            raise MpnError(s, "mpn_step_grads")
        parts, off = [], 0
        for m in self.step_counts:
            parts.append(out[off: off + self.B * m].view(self.B, m))
            off += self.B * m
        return parts

    def mse_grad(self, z, target, g_z=None):
        """dl/dz of the mean squared error of u against target [B][N]."""
        _check_numel("z", z, self.B * self.V * self.N)
        _check_numel("target", target, self.B * self.N)
        if g_z is None:
            g_z = torch.empty_like(z)
        _check_numel("g_z", g_z, self.B * self.V * self.N)
        s = self.lib.mpn_mse_grad(self._h, _ptr(z), _ptr(target), _ptr(g_z), _stream())
        if s != 0:
            raise MpnError(s, "mpn_mse_grad")
        return g_z

    def profile(self, enable=-1):
        """Returns (ms, launches, bytes, kernels): the timed smoothing steps and
        the kernels launched since the last reset; enable=1/0 then switches
        timing on/off and resets."""
        ms, n, by, k = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_double(), ctypes.c_longlong()
        self.lib.mpn_profile(self._h, enable, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(by), ctypes.byref(k))
        return ms.value, n.value, by.value, k.value

    def apply_reduced(self, fields, scalars, u):
        _check_f32("scalars", scalars, (self.V, self.B))
        if self.F > 0:
            _check_f32("fields", fields, (self.F, self.B, self.N))
        _check_numel("u", u, self.B * self.N)
        q = torch.empty_like(u)
        s = self.lib.mpn_apply_reduced(self._h, _ptr(fields) if self.F else None, _ptr(scalars), _ptr(u),
                                       _ptr(q), _stream())
        if s != 0:
            raise MpnError(s, "mpn_apply_reduced")
        return q
