"""Build the CUDA library libhz.so for sm_103a, in tree.

One nvcc process per translation unit (the FFT pass kernels are compiled once
per supported axis length), run in parallel, then linked into
paper_2409_16172_gb300/libhz.so.  Objects go to paper_2409_16172_gb300/_build/.
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
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libhz.so")
FFT_SIZES = (8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 512, 1024, 2048,
             20, 40, 60, 120, 180, 240, 360, 480, 720, 960, 1440, 1920, 2400, 2880, 3600, 4800)
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _units():
    units = []
    for name in ("api.cu", "gmres.cu", "medium.cu", "stencil.cu", "krylov.cu", "profile.cu",
                 "noalloc.cu", "server.cu", "tune.cu"):
        units.append((os.path.join(CSRC, name), os.path.join(OUT, name.replace(".cu", ".o")), []))
    for n in FFT_SIZES:
        units.append((os.path.join(CSRC, "fft_inst.cu"), os.path.join(OUT, f"fft_{n}.o"),
                      [f"-DHZ_FFT_N={n}"]))
    return units


def _sources_digest() -> str:
    h = hashlib.sha256()
    for root in (CSRC, os.path.join(HERE, "..", "include")):
        for f in sorted(os.listdir(root)):
            if f.endswith((".cu", ".cuh", ".h")):
                with open(os.path.join(root, f), "rb") as fh:
                    h.update(f.encode() + fh.read())
    h.update(" ".join(ARCH + FLAGS).encode())
    h.update(platform.machine().encode())
    return h.hexdigest()


def build(force: bool = False, jobs: int | None = None, verbose: bool = False) -> str:
    """Compile every translation unit and link libhz.so; returns its path."""
    os.makedirs(OUT, exist_ok=True)
    stamp = os.path.join(OUT, "stamp")
    digest = _sources_digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as fh:
            if fh.read().strip() == digest:
                return LIB
    cc = nvcc()
    jobs = jobs or max(2, min(len(_units()), os.cpu_count() or 4))

    def compile_one(u):
        src, obj, extra = u
        cmd = [cc] + ARCH + FLAGS + extra + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {os.path.basename(obj)}:\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(jobs) as ex:
        results = list(ex.map(compile_one, _units()))
    if verbose:
        for obj, err in results:
            if err.strip():
                print(obj, err, file=sys.stderr)
    objs = [o for o, _ in results]
    tmp = LIB + ".tmp"
    r = subprocess.run([cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as fh:
        fh.write(digest)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
