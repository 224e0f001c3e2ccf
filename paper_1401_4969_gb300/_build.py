"""In-tree build of libmlev.so for sm_103a (nvcc, no cmake).

Translation units are compiled in parallel and linked into
``paper_1401_4969_gb300/_lib/libmlev.so``. The CUDA runtime is linked statically, so
the library needs only the NVIDIA driver at run time.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "_lib")
LIB = os.path.join(OUT, "libmlev.so")
SOURCES = ["plan.cpp", "kern_mg.cu", "kern_mgfused.cu", "kern_mgreg.cu", "kern_multi.cu", "kern_field.cu", "kern_eig.cu", "kern_adj.cu", "api.cu"]
HEADERS = ["mlev_internal.h", "plan.h", "kern_common.cuh", "kern_launch.h", "kern_blk.cuh", "kern_band.cuh",
           "kern_coarse.cuh", "kern_tail.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O3", "-diag-suppress", "177"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the mlev CUDA library cannot be built")


def _deps():
    return [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(ROOT, "include", "mlev.h"), __file__]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags: list[str] | None = None) -> str:
    """Compile and link libmlev.so if any source is newer; returns the library path."""
    if not force and not extra_flags and up_to_date():
        return LIB
    os.makedirs(os.path.join(OUT, "obj"), exist_ok=True)
    cc = nvcc()
    flags = FLAGS + (extra_flags or [])

    common = [os.path.join(CSRC, f) for f in HEADERS] + [os.path.join(ROOT, "include", "mlev.h"), __file__]
    newest_common = max(os.path.getmtime(d) for d in common)

    def compile_one(src):
        obj = os.path.join(OUT, "obj", src + ".o")
        if (not force and not extra_flags and os.path.exists(obj) and
                os.path.getmtime(obj) >= max(newest_common, os.path.getmtime(os.path.join(CSRC, src)))):
            return obj  # object newer than its source and every header
        cmd = [cc, *ARCH, *flags, "-I", os.path.join(ROOT, "include"), "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
