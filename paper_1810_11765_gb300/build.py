"""Builds the CUDA library ``_lib/libdsoa.so`` in-tree for sm_103a.

Each ``csrc/*.cu`` translation unit is compiled by its own nvcc process (in
parallel) and the objects are linked into one shared library against the shared
CUDA runtime, so that the library and PyTorch use the same runtime instance.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT, "libdsoa.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
         "--expt-relaxed-constexpr", "-I" + INCLUDE, "-I" + CSRC]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdsoa.so")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _fingerprint(extra) -> str:
    h = hashlib.sha256()
    for p in sorted(_sources() + glob.glob(os.path.join(CSRC, "*.cuh")) +
                    glob.glob(os.path.join(INCLUDE, "*.h")) + glob.glob(os.path.join(INCLUDE, "*.cuh"))):
        with open(p, "rb") as f:
            h.update(os.path.relpath(p, ROOT).encode() + b"\0" + f.read())
    h.update(" ".join(ARCH + FLAGS + list(extra)).replace(ROOT, "").encode())
    return h.hexdigest()


def fingerprint(extra_flags=()) -> str:
    """Hash of every CUDA source, header and compile flag of the library."""
    return _fingerprint(extra_flags)


def build(force: bool = False, extra_flags=(), out_lib: str = LIB, verbose: bool = False) -> str:
    """Compile and link; a no-op when sources and flags are unchanged."""
    os.makedirs(OUT, exist_ok=True)
    stamp = out_lib + ".stamp"
    fp = _fingerprint(extra_flags)
    if not force and os.path.exists(out_lib) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == fp:
                return out_lib
    nvcc = _nvcc()
    tag = hashlib.sha256(" ".join(extra_flags).encode()).hexdigest()[:8]
    objs = []
    cmds = []
    for src in _sources():
        obj = os.path.join(OUT, os.path.basename(src)[:-3] + f".{tag}.o")
        objs.append(obj)
        cmds.append([nvcc, *ARCH, *FLAGS, *extra_flags, "-c", src, "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)

    with cf.ThreadPoolExecutor(max_workers=min(len(cmds), os.cpu_count() or 4)) as ex:
        list(ex.map(run, cmds))
    tmp = out_lib + f".tmp{os.getpid()}"
    run([nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs])
    os.replace(tmp, out_lib)
    with open(stamp, "w") as f:
        f.write(fp)
    return out_lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
