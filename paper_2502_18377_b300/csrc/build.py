"""Builds libmpn.so (the C-ABI solver library) for sm_103a with nvcc, and
its bounds-checked variant libmpn_debug.so (-DMPN_DEBUG: the kernels' index
helpers record out-of-range indices in a device word instead of faulting).

Usage: python -m paper_2502_18377_b300.csrc.build [--force] [--debug]
(or call build() / build(debug=True))
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
PKG = os.path.dirname(HERE)
ROOT = os.path.dirname(PKG)
LIB = os.path.join(PKG, "libmpn.so")
LIB_DEBUG = os.path.join(PKG, "libmpn_debug.so")
SOURCES = [os.path.join(HERE, f) for f in ("mpn.cu", "mpn_step_row.cu", "mpn_step_y.cu", "mpn_step_march.cu", "mpn_noalloc.cu",
                                          "mpn_conv.cu")]
DEPS = SOURCES + [os.path.join(HERE, f) for f in os.listdir(HERE) if f.endswith((".cuh", ".h"))] + \
    [os.path.join(ROOT, "include", "mpn.h")]
OBJ_DIR = os.path.join(PKG, "_build")
OBJ_DIR_DEBUG = os.path.join(PKG, "_build_debug")

NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    raise RuntimeError("nvcc not found")


def up_to_date(lib=LIB):
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in DEPS)


def build(force=False, verbose=False, debug=False):
    """Compiles every translation unit to an object in parallel, then links
    the shared library (debug=True: the bounds-checked variant)."""
    lib, obj_dir = (LIB_DEBUG, OBJ_DIR_DEBUG) if debug else (LIB, OBJ_DIR)
    if not force and up_to_date(lib):
        return lib
    from concurrent.futures import ThreadPoolExecutor
    os.makedirs(obj_dir, exist_ok=True)
    inc = ["-I", os.path.join(ROOT, "include")]
    flags = NVCC_FLAGS + (["-DMPN_DEBUG"] if debug else [])

    def compile_one(src):
        obj = os.path.join(obj_dir, os.path.basename(src) + ".o")
        cmd = [nvcc()] + flags + inc + ["-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        return obj, r

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    for obj, r in results:
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + r.stdout + r.stderr)
        if verbose and r.stderr:
            print(r.stderr)
    cmd = [nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-o", lib] + [o for o, _ in results]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc link failed:\n" + r.stdout + r.stderr)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, debug="--debug" in sys.argv)
