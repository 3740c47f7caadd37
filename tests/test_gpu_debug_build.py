"""The bounds-checked build (libmpn_debug.so, compiled with -DMPN_DEBUG):
on small problems that reach every checked index helper, its kernels record
no out-of-range index, and its results equal the release library's.

The debug library runs in a child process (one library per process); the
release results come from this process.  Tolerances: z and d_z relative L2
<= 1e-6 per case (both builds solve to the same tolerance), dl/db <= 1e-5,
the FP32 operator apply <= 1e-6.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
TOL = {"z": 1e-6, "dz": 1e-6, "drhs": 1e-5, "q": 1e-6}


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def test_debug_build_records_no_bad_index_and_matches_release(tmp_path):
    from paper_2502_18377_b300 import binding
    from paper_2502_18377_b300.csrc import build
    lib = build.build(debug=True)
    out = tmp_path / "debug.npz"
    r = subprocess.run([sys.executable, os.path.join(HERE, "_debug_build_cases.py"), lib, str(out)],
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    dbg = dict(np.load(out))
    sys.path.insert(0, HERE)
    import _debug_build_cases as cases
    binding.load()
    rel = cases.run()
    for key, ref in rel.items():
        name, kind = key.split(":")
        if kind == "code":
            assert int(ref) == -1, "the release library reports no index checks"
            assert int(dbg[key]) == 0, f"{name}: out-of-range index, code {int(dbg[key])}"
            continue
        err = _rel(dbg[key], ref)
        assert err <= TOL[kind], (name, kind, err)
