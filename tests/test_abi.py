"""The C-ABI library builds, loads and exports every symbol include/mpn.h
declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mpn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mpn_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_declared_symbols():
    from paper_2502_18377_b300.csrc import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    names = _declared()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


def test_binding_declares_every_export():
    from paper_2502_18377_b300 import binding
    assert sorted(binding.EXPORTS) == _declared()
    binding.load()


def test_error_strings_without_gpu():
    from paper_2502_18377_b300 import binding
    lib = binding.load()
    assert lib.mpn_strerror(0) == b"ok"
    assert b"unsupported" in lib.mpn_strerror(2)
    d = binding.MpnDesc()
    assert lib.mpn_default_desc(ctypes.byref(d)) == 0
    assert d.stencil == 3 and d.inner_iters >= 1
    assert d.fused_coarse == 1 and d.fused_step == 3 and d.krylov == 0 and d.coarsen_time == 0 and d.direct == 0 and d.max_coarse == 2048   # last fields: layout agrees with the header
    assert lib.mpn_fused_level(None) == -1
    h = ctypes.c_void_p()
    d.stencil = 5
    assert lib.mpn_create(ctypes.byref(d), ctypes.byref(h)) == 2      # five-point rows: unsupported
    d.stencil = 3
    d.periodic[0] = 1
    assert lib.mpn_create(ctypes.byref(d), ctypes.byref(h)) == 1      # periodic time: invalid
    d.periodic[0] = 0
    d.krylov = 7
    assert lib.mpn_create(ctypes.byref(d), ctypes.byref(h)) == 1      # unknown inner solver: invalid
    d.krylov = 0
    d.batch = 65536
    assert lib.mpn_create(ctypes.byref(d), ctypes.byref(h)) == 2      # more instances than a grid extent: unsupported
    d.batch = 1
    assert d.adj_inner_iters == 0                                     # the last field: the adjoint's own count unset
    d.adj_inner_iters = -1
    assert lib.mpn_create(ctypes.byref(d), ctypes.byref(h)) == 1      # negative iteration count: invalid


def test_binding_rejects_missized_tensors_without_launching():
    """The allocation-free apply takes its sizes from a descriptor built apart
    from the tensors: a short output, a short operand or a non-float32 tensor
    is refused on the host, before anything reaches the library (CPU tensors:
    nothing here can launch)."""
    import pytest
    import torch
    from paper_2502_18377_b300 import binding
    geom = dict(n=(8, 16, 16), step=(1 / 7, 1 / 16, 1 / 16), periodic=(False, True, True))
    desc = binding.make_desc(geom, 2, [1, -1, -1, -1, 0, -1, 0], 2)
    N = 8 * 16 * 16
    ok = dict(fields=torch.zeros(2, 2, N), scalars=torch.zeros(7, 2), u=torch.zeros(2, N), q=torch.zeros(2, N))
    for name, bad in (("q", torch.zeros(2, N - 1)), ("u", torch.zeros(N)), ("fields", torch.zeros(1, 2, N)),
                      ("scalars", torch.zeros(7, 1)), ("u", torch.zeros(2, N, dtype=torch.float64))):
        args = dict(ok)
        args[name] = bad
        with pytest.raises(ValueError, match=name):
            binding.apply_reduced_noalloc(desc, args["fields"], args["scalars"], args["u"], args["q"])


def test_noalloc_refuses_operators_it_does_not_apply():
    """The allocation-free apply implements uniform steps and Dirichlet faces
    only: per-interval steps and Neumann / mixed rows are refused with
    UNSUPPORTED, and a face with alpha = beta = 0 with INVALID_ARG, by the
    host-side checks before any launch (the pointers are never used)."""
    from paper_2502_18377_b300 import binding
    lib = binding.load()
    geom = dict(n=(8, 16, 16), step=(1 / 7, 1 / 15, 1 / 16), periodic=(False, False, True))
    fake = ctypes.c_void_p(256)
    call = lambda d: lib.mpn_apply_reduced_noalloc(ctypes.byref(d), fake, fake, fake, fake, None)
    d = binding.make_desc(geom, 2, [1, -1, -1, -1, 0, -1, 0], 2)
    d.variable_steps = 1
    assert call(d) == 2
    d = binding.make_desc(geom, 2, [1, -1, -1, -1, 0, -1, 0], 2)
    d.bc_alpha[1], d.bc_beta[1] = 1.0, 0.5
    assert call(d) == 2
    d.bc_alpha[1], d.bc_beta[1] = 0.0, 0.0
    assert call(d) == 1


def test_unaligned_arrays_are_refused_before_any_launch():
    """The operator and convolution kernels move 16-byte pieces: an array
    argument that is not 16-byte aligned is refused with INVALID_ARG by the
    host-side checks, before the problem object or any pointer is used."""
    from paper_2502_18377_b300 import binding
    lib = binding.load()
    ok, odd = ctypes.c_void_p(4096), ctypes.c_void_p(4096 + 4)
    fake_problem = ctypes.c_void_p(64)   # never dereferenced: the check comes first
    assert lib.mpn_apply_reduced(fake_problem, ok, ok, odd, ok, None) == 1
    assert lib.mpn_apply_reduced(fake_problem, ok, ok, ok, odd, None) == 1
    d = binding.MpnConvDesc()
    for k in range(3):
        d.n[k], d.periodic[k] = 8, int(k > 0)
    d.batch, d.cin, d.cout = 1, 32, 32
    assert lib.mpn_conv3d_forward(ctypes.byref(d), odd, ok, None, ok, 0, None) == 1
    assert lib.mpn_conv3d_forward(ctypes.byref(d), ok, ok, None, odd, 0, None) == 1
    assert lib.mpn_conv3d_backward_data(ctypes.byref(d), ok, ok, odd, ok, None) == 1
    assert lib.mpn_conv3d_backward_weights(ctypes.byref(d), ok, odd, ok, ok, ok, None) == 1


def test_solver_rejects_missized_tensors_without_launching():
    """The solve, the adjoint and the loss gradient read and write B*V*N (or
    B*N) values through raw pointers: a tensor of another size or dtype is
    refused on the host before the library is called (CPU tensors and a
    Solver without a problem object: nothing here can reach a GPU)."""
    import pytest
    import torch
    from paper_2502_18377_b300.binding import Solver
    s = object.__new__(Solver)
    s.B, s.V, s.N, s.F = 2, 7, 64, 2
    args = (torch.zeros(2, 2, 64), torch.zeros(7, 2), torch.zeros(2, 64), torch.zeros(2, 64))
    with pytest.raises(ValueError, match="u0"):
        s.forward(*args, u0=torch.zeros(2, 63))
    with pytest.raises(ValueError, match="z"):
        s.forward(*args, z=torch.zeros(2, 7, 63))
    with pytest.raises(ValueError, match="z64"):
        s.forward(*args, z64=torch.zeros(2, 7, 64))            # float32, not float64
    with pytest.raises(ValueError, match="z"):
        s.adjoint(*args, torch.zeros(2, 6, 64), torch.zeros(2, 7, 64))
    with pytest.raises(ValueError, match="target"):
        s.mse_grad(torch.zeros(2, 7, 64), torch.zeros(2, 65))
    with pytest.raises(ValueError, match="g_z"):
        s.mse_grad(torch.zeros(2, 7, 64), torch.zeros(2, 64), g_z=torch.zeros(2, 7, 64, dtype=torch.float64))


def test_benchmark_settings_are_solver_options():
    """Every benchmark workload's solver settings name options the solver
    takes, with values the descriptor accepts (iteration counts >= 1, the
    adjoint's >= 0, degrees 1..30), so the benchmark, the profiling driver
    and the full-size tests cannot fail on a misspelt or invalid setting."""
    import inspect
    from paper_2502_18377_b300 import settings
    from paper_2502_18377_b300.binding import Solver
    params = inspect.signature(Solver.__init__).parameters
    for name, (gen, batch, grid, seed, kw) in settings.BENCH_WORKLOADS.items():
        assert callable(gen) and batch >= 1 and all(n >= 8 for n in grid), name
        for k, v in kw.items():
            assert k in params, (name, k)
        assert kw.get("inner_iters", 5) >= 1 and kw.get("adj_inner_iters", 0) >= 0, name
        assert 1 <= kw.get("cheb_degree", 5) <= 30, name
