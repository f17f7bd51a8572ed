"""Builds libuhnsw.so in-tree: every .cu file with nvcc for sm_103a and the
host graph builder with g++, compiled in parallel, linked with nvcc."""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INC = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libuhnsw.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")
# UHNSW_CHECK=1 builds the diagnostic variant whose kernels record (and clamp)
# any out-of-range index instead of accessing it.
CHECK = os.environ.get("UHNSW_CHECK", "0") == "1"
EXTRA = ["-DUHNSW_CHECK"] if CHECK else []
# extra nvcc flags for tuning builds, e.g. UHNSW_NVCC_EXTRA="-DUHNSW_WARP_MINB=10"
EXTRA += os.environ.get("UHNSW_NVCC_EXTRA", "").split()


def _sources():
    cu = sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))
    cpp = sorted(f for f in os.listdir(CSRC) if f.endswith(".cpp"))
    deps = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC)) + [os.path.join(INC, "uhnsw.h")]
    return cu, cpp, deps


def _compile(src: str) -> str:
    obj = os.path.join(OUT_DIR, src.rsplit(".", 1)[0] + ".o")
    path = os.path.join(CSRC, src)
    if src.endswith(".cu"):
        cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", *EXTRA,
               f"-I{INC}", f"-I{CSRC}", "-c", path, "-o", obj]
    else:
        cmd = ["g++", "-O3", "-std=c++17", "-fPIC", "-pthread", f"-I{INC}", f"-I{CSRC}",
               "-I/usr/local/cuda/include", "-c", path, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return obj


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    cu, cpp, deps = _sources()
    newest = max(os.path.getmtime(p) for p in deps)
    stamp = LIB + ".flags"
    flags = " ".join(EXTRA)
    same_flags = os.path.exists(stamp) and open(stamp).read() == flags
    if not force and same_flags and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    srcs = cu + cpp
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 4))) as ex:
        objs = list(ex.map(_compile, srcs))
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-fPIC", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(flags)
    if verbose:
        print(LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
