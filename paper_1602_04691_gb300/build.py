"""Build the CUDA library libori.so in-tree for sm_103a.

The translation units are compiled in parallel with nvcc and linked against
the shared CUDA runtime (the same libcudart PyTorch loads).  The FFT passes are
compiled as twelve units, one per arithmetic and part (passes_inst.cu with
ORI_PASS_T / ORI_PASS_PART), since their template instances dominate the
build time.  A stamp
of the sources and flags skips the build when nothing changed.
"""

from __future__ import annotations

import glob
import hashlib
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libori.so")

SOURCES = ["ori_api.cu", "ori_noalloc.cu", "passes_inst.cu"]
# (object name, source, extra flags): passes_inst.cu once per arithmetic T and part
UNITS = [("ori_api", "ori_api.cu", []), ("ori_noalloc", "ori_noalloc.cu", [])] + [
    (f"passes_{tn}_{pn}", "passes_inst.cu", [f"-DORI_PASS_T={ti}", f"-DORI_PASS_PART={pi}"])
    for ti, tn in ((1, "f32"), (2, "f64"), (3, "df")) for pi, pn in ((1, "x"), (2, "yfwd"), (3, "yinv"), (4, "z"))]
# Every header next to the sources is part of the stamp, so an edit to any of them rebuilds.
HEADERS = sorted(os.path.basename(f) for f in glob.glob(os.path.join(CSRC, "*.cuh")))
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
         "-I" + os.path.join(ROOT, "include")]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def stamped_files() -> list[str]:
    """Absolute paths of every file whose contents enter the build stamp."""
    return [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(ROOT, "include", "ori.h")]


def _stamp() -> str:
    h = hashlib.sha256()
    for path in stamped_files():
        with open(path, "rb") as fh:
            h.update(os.path.basename(path).encode() + fh.read())
    h.update(" ".join(ARCH + FLAGS).encode())
    h.update(repr(UNITS).encode())
    h.update(os.uname().machine.encode())
    return h.hexdigest()


def build(verbose: bool = False, force: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    stamp = _stamp()
    stamp_file = os.path.join(BUILD, "libori.stamp")
    if not force and os.path.exists(LIB) and os.path.exists(stamp_file):
        with open(stamp_file) as fh:
            if fh.read().strip() == stamp:
                return LIB
    nvcc = _nvcc()

    def compile_one(unit) -> str:
        name, src, extra = unit
        obj = os.path.join(BUILD, name + ".o")
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed for {name}:\n{res.stdout}\n{res.stderr}")
        return obj

    with ThreadPoolExecutor(max_workers=min(len(UNITS), max(2, os.cpu_count() or 2))) as ex:
        objs = list(ex.map(compile_one, UNITS))
    tmp = LIB + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, LIB)
    with open(stamp_file, "w") as fh:
        fh.write(stamp)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
