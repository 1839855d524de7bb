"""Build the CPU oracle shared library (test infrastructure).

gcc, -O2, no FP contraction (a*b+c must stay two rounded operations so that
strict mode matches the GPU built with --fmad=false), no fast-math.  The output
goes to oracle/_build/liboracle.so and is rebuilt when a source is newer.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["rng.c", "specmath.c", "tables.c", "transport.c"]
HEADERS = ["oracle.h", "transport_body.h"]
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-pthread",
          "-Wall", "-Wno-unused-function", "-D_GNU_SOURCE"]


def build(force: bool = False) -> str:
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    deps = srcs + [os.path.join(HERE, h) for h in HEADERS]
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= t for d in deps):
            return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", *CFLAGS, "-shared", "-o", tmp, *srcs, "-lm"]
    subprocess.run(cmd, check=True, cwd=HERE)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
