"""In-tree build of the CUDA library (``_build/libadvect.so``) for sm_103a.

Each ``csrc/*.cu`` file is compiled by nvcc in parallel and linked into one
shared library exporting the C ABI of ``include/advect.h``.  The roofline
probe (``probe/*.cu``: the binary64 pipe's throughput, measured by the
benchmark) is linked into a library of its own, ``_build/libadvect_probe.so``.
The build is skipped when a stamp of the sources and flags is unchanged.
"""
from __future__ import annotations

import concurrent.futures as cf
import fcntl
import glob
import hashlib
import os
import platform
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libadvect.so")
PROBE = os.path.join(HERE, "probe")
PROBE_LIB = os.path.join(BUILD, "libadvect_probe.so")
NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
                "--expt-relaxed-constexpr", "-Xptxas", "-v"]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _probe_sources():
    return sorted(glob.glob(os.path.join(PROBE, "*.cu")))


def _stamp() -> str:
    h = hashlib.sha1()
    files = _sources() + sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")))
    files += _probe_sources()
    files.append(os.path.join(ROOT, "include", "advect.h"))
    for f in files:
        h.update(f.encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(FLAGS).encode())
    h.update(platform.machine().encode())
    return h.hexdigest()


def _up_to_date(stamp: str) -> bool:
    stamp_path = os.path.join(BUILD, "stamp")
    if not (os.path.exists(LIB) and os.path.exists(PROBE_LIB) and os.path.exists(stamp_path)):
        return False
    with open(stamp_path) as f:
        return f.read().strip() == stamp


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link the library if sources changed; returns its path.
    Processes that build at the same time (one per rank) serialise on a lock
    file; the ones that wait find the library up to date."""
    stamp = _stamp()
    if not force and _up_to_date(stamp):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    with open(os.path.join(BUILD, "lock"), "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)
        try:
            if not force and _up_to_date(stamp):
                return LIB
            return _compile_and_link(stamp, verbose)
        finally:
            fcntl.flock(lock, fcntl.LOCK_UN)


def _compile_and_link(stamp: str, verbose: bool) -> str:
    stamp_path = os.path.join(BUILD, "stamp")
    obj_dir = os.path.join(BUILD, "obj")
    os.makedirs(obj_dir, exist_ok=True)

    def compile_one(src):
        obj = os.path.join(obj_dir, os.path.basename(src)[:-3] + ".o")
        cmd = [NVCC, *FLAGS, "-I", os.path.join(ROOT, "include"), "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    srcs = _sources()
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        results = list(ex.map(compile_one, srcs + _probe_sources()))
    if verbose:
        for obj, log in results:
            print(f"== {os.path.basename(obj)}\n{log}")
    objs = [o for o, _ in results]
    for lib, parts in ((LIB, objs[:len(srcs)]), (PROBE_LIB, objs[len(srcs):])):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *parts]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    with open(stamp_path, "w") as f:
        f.write(stamp)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
