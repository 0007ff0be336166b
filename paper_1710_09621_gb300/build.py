"""Build the in-tree CUDA shared library libodwf.so for sm_103a (GB300).

Each translation unit under csrc/ is compiled by its own nvcc process in parallel, then linked
with the CUDA runtime. The library is written next to this file so that it is loaded from the
source tree, not from site-packages.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import platform
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libodwf.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["kernels.cu", "eofa.cu", "solver.cpp", "api.cpp", "noalloc.cu", "learned.cu", "hmc.cu", "hop_pair.cu", "peak.cu"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags():
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
                   "--expt-relaxed-constexpr"]


def _compile(src: str) -> str:
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc()] + _flags() + ["-x", "cu", "-c", os.path.join(CSRC, src), "-o", obj]
    if os.environ.get("ODWF_PTXAS_VERBOSE"):
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if os.environ.get("ODWF_PTXAS_VERBOSE"):
        sys.stderr.write(r.stderr)
    return obj


STAMP = LIB + ".stamp"


def source_hash() -> str:
    """SHA-256 over every source and header, the compile flags, the source list and the host
    architecture: the library is rebuilt whenever any of them differs from the one it was built from
    (file times are not used, so a library copied in from elsewhere is never mistaken for current)."""
    hs = hashlib.sha256()
    hs.update(platform.machine().encode())
    hs.update(" ".join(_flags() + SOURCES).replace(ROOT, "<root>").encode())
    for d in (CSRC, INCLUDE):
        for f in sorted(os.listdir(d)):
            fp = os.path.join(d, f)
            if os.path.isfile(fp):
                hs.update(f.encode())
                with open(fp, "rb") as fh:
                    hs.update(fh.read())
    return hs.hexdigest()


def _stale() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(STAMP):
        return True
    with open(STAMP) as fh:
        return fh.read().strip() != source_hash()


def build(force: bool = False) -> str:
    """Compile csrc/*.cu and csrc/*.cpp into libodwf.so; returns the library path."""
    if not force and not _stale():
        return LIB
    # the hash of the sources as they are when the compile starts: a source edited while it runs
    # leaves the library stale for the next call
    digest = source_hash()
    os.makedirs(BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(_compile, SOURCES))
    tmp = LIB + ".tmp"
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(STAMP, "w") as fh:
        fh.write(digest + "\n")
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
