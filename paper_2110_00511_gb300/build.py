"""Builds libash.so (the C ABI of include/ash.h) for sm_103a with nvcc.

Translation units compile in parallel: the map host code, the
dimension-independent kernels, and one instantiation of the map kernels per
key dimension 1..8.  Output: paper_2110_00511_gb300/_lib/libash.so (git-ignored).
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OBJ = os.path.join(PKG, "_build")
LIBDIR = os.path.join(PKG, "_lib")
LIB = os.path.join(LIBDIR, "libash.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + os.path.join(ROOT, "include"), "-I" + CSRC]


def _nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found")
    return exe


def _units():
    units = [("ash_map.cu", []), ("ash_aux.cu", []), ("ash_trace.cu", []), ("ash_batch.cu", []), ("ash_tune.cu", []), ("ash_server.cu", []), ("ash_replay.cu", []),
             ("ash_volume.cu", [])]
    units += [("ash_dim.cu", [f"-DASH_DIM={d}"]) for d in range(1, 9)]
    return units


def _sources():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "ash.h"), __file__]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OBJ, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(unit):
        src, defs = unit
        tag = os.path.splitext(src)[0] + "".join(d.replace("-D", "_").replace("=", "") for d in defs)
        out = os.path.join(OBJ, tag + ".o")
        cmd = [nvcc, *ARCH, *FLAGS, *extra_flags, *defs, "-c", os.path.join(CSRC, src), "-o", out]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src} {defs}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return out

    with cf.ThreadPoolExecutor(max_workers=min(10, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, _units()))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                extra_flags=["-Xptxas", "-v"] if "--ptxas" in sys.argv else []))
