"""Build libbldtt.so in-tree with nvcc for sm_103a (GB300).

Each translation unit is compiled in parallel, then linked into a shared
library next to this file.  A stamp of the sources and flags skips rebuilds
when nothing changed.  build_pipes() builds the benchmark's separate
pipe-throughput library (libbldtt_pipes.so) from csrc_bench/.
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(HERE, "libbldtt.so")

SOURCES = ["prims.cu", "tree.cu", "dtt.cu", "passes.cu", "interact.cu", "direct.cu", "capi.cu",
           "noalloc.cu", "learned.cu", "waitprobe.cu", "shard.cu", "passes_tc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
                 "--expt-relaxed-constexpr", f"-I{INCLUDE}"]
# Geometric decisions (tree splits, MAC) must be plain FP64 expressions.
PER_FILE = {"tree.cu": ["-fmad=false"], "dtt.cu": ["-fmad=false"]}


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libbldtt.so")


def _stamp(extra_flags) -> str:
    h = hashlib.sha256()
    for name in sorted(os.listdir(CSRC)):
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(name.encode() + f.read())
    with open(os.path.join(INCLUDE, "bldtt.h"), "rb") as f:
        h.update(f.read())
    h.update(" ".join(COMMON + list(extra_flags)).encode())
    h.update(repr(sorted(PER_FILE.items())).encode())
    return h.hexdigest()


def build(verbose: bool = False, force: bool = False, extra_flags=()) -> str:
    """Compile and link libbldtt.so; returns its path."""
    stamp = _stamp(extra_flags)
    stamp_path = os.path.join(BUILD_DIR, "stamp")
    if not force and os.path.exists(LIB_PATH) and os.path.exists(stamp_path):
        with open(stamp_path) as f:
            if f.read().strip() == stamp:
                return LIB_PATH
    os.makedirs(BUILD_DIR, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD_DIR, src.replace(".cu", ".o"))
        cmd = [nvcc, *COMMON, *PER_FILE.get(src, []), *extra_flags, "-c",
               os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, flush=True)
        return obj

    with ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB_PATH + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB_PATH)
    with open(stamp_path, "w") as f:
        f.write(stamp)
    return LIB_PATH


PIPES_SRC = os.path.join(HERE, "csrc_bench", "pipes.cu")
PIPES_LIB = os.path.join(HERE, "libbldtt_pipes.so")


def build_pipes(force: bool = False) -> str:
    """Compile the pipe microbenchmark used by bench.py (not part of
    libbldtt.so); returns the library's path."""
    h = hashlib.sha256()
    with open(PIPES_SRC, "rb") as f:
        h.update(f.read())
    h.update(" ".join(ARCH).encode())
    stamp = h.hexdigest()
    stamp_path = os.path.join(BUILD_DIR, "pipes.stamp")
    if not force and os.path.exists(PIPES_LIB) and os.path.exists(stamp_path):
        with open(stamp_path) as f:
            if f.read().strip() == stamp:
                return PIPES_LIB
    os.makedirs(BUILD_DIR, exist_ok=True)
    tmp = PIPES_LIB + ".tmp"
    cmd = [_nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
           PIPES_SRC, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on csrc_bench/pipes.cu:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, PIPES_LIB)
    with open(stamp_path, "w") as f:
        f.write(stamp)
    return PIPES_LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
