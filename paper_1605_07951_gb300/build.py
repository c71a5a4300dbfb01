"""In-tree build of librsrr.so (sm_103a) with nvcc, translation units in parallel."""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "librsrr.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I" + os.path.join(ROOT, "include"), "-I" + CSRC]

# (source, extra flags, object name)
UNITS = [
    ("api.cu", [], "api.o"),
    ("band.cu", [], "band.o"),
    ("band_lu.cu", ["-DRSRR_LU_ONLY=64"], "band_lu64.o"),
    ("band_lu.cu", ["-DRSRR_LU_ONLY=128"], "band_lu128.o"),
    ("band_lu.cu", ["-DRSRR_LU_ONLY=32"], "band_lu_r32.o"),
    ("band_lu.cu", ["-DRSRR_LU_ONLY=65"], "band_lu_r64.o"),
    ("proj.cu", [], "proj.o"),
    ("ssfull_host.cpp", ["-x", "cu", "-Xcompiler", "-fcx-fortran-rules"], "ssfull_host.o"),
    ("noalloc.cu", [], "noalloc.o"),
    ("dense.cu", [], "dense.o"),
    ("dense_tc.cu", [], "dense_tc.o"),
    ("refine.cu", [], "refine.o"),
    ("ozaki.cu", [], "ozaki.o"),
    ("band_solve2.cu", [], "band_solve2.o"),
    ("server.cu", [], "server.o"),
    ("ssfull_dev.cu", [], "ssfull_dev.o"),
]


def nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _compile(unit):
    src, extra, obj = unit
    out = os.path.join(OUT_DIR, obj)
    cmd = [nvcc()] + ARCH + FLAGS + extra + ["-c", os.path.join(CSRC, src), "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return out


def build(verbose: bool = False) -> str:
    """Compile every CUDA translation unit for sm_103a and link librsrr.so."""
    os.makedirs(OUT_DIR, exist_ok=True)
    units = [u for u in UNITS if os.path.exists(os.path.join(CSRC, u[0]))]
    with ThreadPoolExecutor(max_workers=max(1, min(len(units), os.cpu_count() or 1))) as ex:
        objs = list(ex.map(_compile, units))
    tmp = LIB + ".tmp"
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-cudart", "shared", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        print("built", LIB, file=sys.stderr)
    return LIB


if __name__ == "__main__":
    build(verbose=True)
