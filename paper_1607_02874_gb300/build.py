"""Build liblbm.so in-tree for sm_103a with nvcc (no cmake, parallel units)."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "liblbm.so")
# the bounds-checked debugging build (-DLBM_CHECKED)
CHECKED_DIR = os.path.join(HERE, "_lib_checked")
CHECKED_LIB = os.path.join(CHECKED_DIR, "liblbm.so")
UNITS = ["capi.cu", "geometry.cu", "observe_noalloc.cu", "halo.cu"] + [
    f"step_{st}{mode}.cu" for mode in ("", "_rs", "_bary", "_rs_bary", "_chan", "_rs_chan") for st in ("f32", "f16", "bf16")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-fopenmp,-O3", "--expt-relaxed-constexpr"]
# the checked build optimises device code lightly: it compiles 5x faster, and
# its speed does not matter
CHECKED_FLAGS = ["-DLBM_CHECKED", "-Xcicc", "-O1", "-Xptxas", "-O1"]


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(os.path.dirname(HERE), "include", "lbm.h"))
    files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compile every unit to an object and link the shared library (with
    checked=True the bounds-checked debugging build, in its own folder)."""
    out_dir, lib = (CHECKED_DIR, CHECKED_LIB) if checked else (OUT_DIR, LIB)
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _deps():
        return lib
    os.makedirs(out_dir, exist_ok=True)
    # objects are intermediates: compiled into a scratch folder, removed after linking
    obj_dir = tempfile.mkdtemp(prefix="obj", dir=out_dir)

    def compile_unit(u):
        obj = os.path.join(obj_dir, u + ".o")
        cmd = [NVCC, *ARCH, *FLAGS, *(CHECKED_FLAGS if checked else []), "-c", os.path.join(CSRC, u), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {u}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    try:
        with ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
            objs = list(ex.map(compile_unit, UNITS))
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [NVCC, *ARCH, "-shared", "-Xcompiler", "-fopenmp", "-o", tmp, *objs, "-lgomp"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, lib)
    finally:
        shutil.rmtree(obj_dir, ignore_errors=True)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, checked="--checked" in sys.argv))
