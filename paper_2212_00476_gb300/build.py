"""Builds libzncc.so in-tree for sm_103a: every translation unit in parallel, then one link.

    python -m paper_2212_00476_gb300.build [--force] [--verbose-ptxas]

The window radius is a template parameter of the ZNCC kernel; zncc_row.cu is compiled once
per radius 1..7 (window sides 3..15) so that the seven objects build concurrently.
"""

from __future__ import annotations

import argparse
import concurrent.futures as cf
import glob
import hashlib
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libzncc.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
RADII = range(1, 8)


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libzncc.so")


def _units():
    """(source, object, extra flags) for every translation unit."""
    units = [(os.path.join(CSRC, "api.cu"), "api.o", []),
             (os.path.join(CSRC, "kernels.cu"), "kernels.o", []),
             (os.path.join(CSRC, "static_scratch.cu"), "static_scratch.o", []),
             (os.path.join(CSRC, "plane.cu"), "plane.o", []),
             (os.path.join(CSRC, "serve.cpp"), "serve.o", [])]
    for r in RADII:
        units.append((os.path.join(CSRC, "zncc_row.cu"), f"zncc_row_r{r}.o", [f"-DZNCC_R={r}"]))
    return units


def _sources_digest() -> str:
    h = hashlib.sha256()
    for p in sorted(glob.glob(os.path.join(CSRC, "*")) + [os.path.join(INCLUDE, "zncc.h"), __file__]):
        with open(p, "rb") as f:
            h.update(os.path.basename(p).encode())
            h.update(f.read())
    return h.hexdigest()


def build(force: bool = False, verbose_ptxas: bool = False, jobs: int | None = None) -> str:
    digest = _sources_digest()
    stamp = os.path.join(BUILD, "digest")
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == digest:
                return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    common = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
              "-I", INCLUDE, "-I", CSRC, "--expt-relaxed-constexpr"]
    if verbose_ptxas:
        common += ["-Xptxas", "-v"]

    def compile_one(u):
        src, obj, extra = u
        out = os.path.join(BUILD, obj)
        cmd = [*common, *extra, "-c", src, "-o", out]
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed for {obj}:\n{' '.join(cmd)}\n{p.stdout}{p.stderr}")
        return out, p.stdout + p.stderr

    units = _units()
    jobs = jobs or min(len(units), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(jobs) as ex:
        results = list(ex.map(compile_one, units))
    if verbose_ptxas:
        for _, log in results:
            sys.stderr.write(log)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *[o for o, _ in results]]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"link failed:\n{' '.join(cmd)}\n{p.stdout}{p.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(digest)
    return LIB


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--verbose-ptxas", action="store_true")
    args = ap.parse_args()
    print(build(force=args.force, verbose_ptxas=args.verbose_ptxas))
