"""Build the CUDA library libet.so in-tree for sm_103a.

Sixteen kernel objects (strict/fast mode x the eight track layouts) from one
source, the C ABI host objects and the table builder, compiled in
parallel and linked into paper_2302_08252_gb300/_build/libet.so.  Strict
objects use --fmad=false with IEEE division/square root and no flush to zero;
host code uses -ffp-contract=off (the toy model fixes every rounding).
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import re
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INC = os.path.join(ROOT, "include")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libet.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return p


COMMON = ["-std=c++17", *ARCH, "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler",
          "-ffp-contract=off", "-I", INC, "-I", CSRC]
STRICT = ["--fmad=false", "-prec-div=true", "-prec-sqrt=true", "-ftz=false"]
FAST = ["-ftz=false"]


def _sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC)) + sorted(
        os.path.join(INC, f) for f in os.listdir(INC))


def _fingerprint() -> str:
    h = hashlib.sha256()
    for p in _sources():
        with open(p, "rb") as f:
            h.update(p.encode())
            h.update(f.read())
    flags = [f for f in COMMON if f not in (INC, CSRC)] + STRICT + FAST  # no machine paths
    h.update(" ".join(flags).encode())
    return h.hexdigest()


# The sources the transport kernels (kernels_tu.cu) are compiled from.
KERNEL_SOURCES = ("kernels_tu.cu", "kernels.cuh", "physics.cuh", "layout.cuh", "common.cuh",
                  "registry.h")


def _code_only(text: str) -> str:
    """C++ source without comments and whitespace (what the compiler sees)."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return re.sub(r"\s+", "", text)


def kernel_fingerprint() -> str:
    """Hash of the transport kernels' code (comments and whitespace removed) and flags: a
    profile taken on one build stays valid while this is unchanged (host-side code and
    comments may change)."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(CSRC, name), encoding="utf-8") as f:
            h.update(name.encode())
            h.update(_code_only(f.read()).encode())
    flags = [f for f in COMMON if f not in (INC, CSRC)] + STRICT + FAST  # no machine paths
    h.update(" ".join(flags).encode())
    return h.hexdigest()


def _jobs():
    jobs = []
    for mode in (0, 1):
        for layout in range(8):
            obj = os.path.join(OUT, f"k_{mode}_{layout}.o")
            flags = STRICT if mode == 0 else FAST
            jobs.append([_nvcc(), *COMMON, *flags, f"-DET_MODE={mode}", f"-DET_LAYOUT={layout}",
                         "-c", os.path.join(CSRC, "kernels_tu.cu"), "-o", obj])
    jobs.append([_nvcc(), *COMMON, *STRICT, "-c", os.path.join(CSRC, "et_api.cu"), "-o",
                 os.path.join(OUT, "et_api.o")])
    jobs.append([_nvcc(), *COMMON, *STRICT, "-c", os.path.join(CSRC, "noalloc.cu"), "-o",
                 os.path.join(OUT, "noalloc.o")])
    jobs.append([_nvcc(), *COMMON, *STRICT, "-c", os.path.join(CSRC, "fp64.cu"), "-o",
                 os.path.join(OUT, "fp64.o")])
    jobs.append(["g++", "-std=c++17", "-O2", "-fPIC", "-ffp-contract=off", "-I", INC, "-c",
                 os.path.join(CSRC, "toy_tables.cpp"), "-o", os.path.join(OUT, "toy_tables.o")])
    return jobs


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    stamp = os.path.join(OUT, "libet.fingerprint")
    fp = _fingerprint()
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == fp:
                return LIB
    jobs = _jobs()
    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
        futs = [ex.submit(subprocess.run, j, capture_output=True, text=True) for j in jobs]
        for j, fu in zip(jobs, futs):
            r = fu.result()
            if r.returncode != 0:
                raise RuntimeError(f"build failed: {' '.join(j)}\n{r.stdout}\n{r.stderr}")
            if verbose and r.stderr:
                print(r.stderr)
    objs = [j[j.index("-o") + 1] for j in jobs]
    tmp = LIB + f".tmp{os.getpid()}"
    link = [_nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(link)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(fp)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True))
