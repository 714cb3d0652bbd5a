"""Builds the sm_103a shared library ``libfcn_gb300.so`` in-tree.

Each ``csrc/*.cu`` translation unit is compiled by nvcc in parallel into
``_build/`` and then linked (CUDA runtime linked statically) next to this file.
The build is incremental by content: every object carries a key (SHA-256 of
its source, every header, the flags, the nvcc version and the host machine
type) and is recompiled when the key differs, so an object compiled on
another machine, by another compiler or from other sources is never linked.
``build()`` reports how many units it compiled.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import platform
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(ROOT, "_build", "fcn")
LIB = os.path.join(HERE, "libfcn_gb300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]
if os.environ.get("FCN_CHECKED") == "1":      # self-checking kernels (range checks)
    FLAGS.append("-DFCN_CHECKED")
    BUILD = BUILD + "_checked"


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
                  + glob.glob(os.path.join(ROOT, "include", "*.h")))


_NVCC_VERSION = None


def _nvcc_version() -> str:
    global _NVCC_VERSION
    if _NVCC_VERSION is None:
        _NVCC_VERSION = subprocess.run([nvcc(), "--version"], capture_output=True,
                                       text=True).stdout
    return _NVCC_VERSION


def _key(src: str) -> str:
    h = hashlib.sha256()
    h.update(" ".join(ARCH + FLAGS).encode())
    h.update(_nvcc_version().encode())
    h.update(platform.machine().encode())
    for p in [src] + _headers():
        h.update(os.path.basename(p).encode())
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def _read(path: str) -> str:
    try:
        with open(path) as f:
            return f.read().strip()
    except OSError:
        return ""


def _compile(src: str):
    obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
    key = _key(src)
    if os.path.exists(obj) and _read(obj + ".key") == key:
        return obj, False
    cmd = [nvcc()] + ARCH + FLAGS + ["-c", src, "-o", obj + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    os.replace(obj + ".tmp", obj)
    with open(obj + ".key", "w") as f:
        f.write(key)
    return obj, True


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    if force:
        for o in glob.glob(os.path.join(BUILD, "*.o")):
            os.remove(o)
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 4))) as ex:
        res = list(ex.map(_compile, srcs))
    objs = [o for o, _ in res]
    ncomp = sum(1 for _, c in res if c)
    h = hashlib.sha256()
    for o in objs:
        h.update(_read(o + ".key").encode())
    lib_key = h.hexdigest()
    linked = False
    if force or ncomp or not os.path.exists(LIB) or _read(LIB + ".key") != lib_key:
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = [nvcc()] + ARCH + ["-shared", "-Xcompiler", "-fPIC", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
        with open(LIB + ".key", "w") as f:
            f.write(lib_key)
        linked = True
    if verbose:
        print(f"built {LIB} on {platform.machine()}: compiled {ncomp} of {len(srcs)} units, "
              f"{'linked' if linked else 'up to date'}", file=sys.stderr)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
