"""Compile the C oracle into shared libraries beside its source.

Two builds of the same file: a single-threaded one and an OpenMP one (only
element-wise loops are parallel there, so both give identical bytes).
Test infrastructure only.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "gbsz_oracle.c")
LIB = os.path.join(HERE, "libgbsz_oracle.so")
LIB_OMP = os.path.join(HERE, "libgbsz_oracle_omp.so")

# -ffp-contract=off: no fused multiply-add (gcc contracts by default on Arm);
# no fast-math: every float operation stays one IEEE round-to-nearest step.
CFLAGS = ["-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
          "-shared", "-Wall", "-Wno-unknown-pragmas", "-Wno-maybe-uninitialized"]


def _stale(lib):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(os.path.join(HERE, f)) > t
               for f in ("gbsz_oracle.c", "gbsz_oracle.h"))


def build(force=False, verbose=False):
    jobs = []
    if force or _stale(LIB):
        jobs.append(["gcc", *CFLAGS, SRC, "-o", LIB, "-lm"])
    if force or _stale(LIB_OMP):
        jobs.append(["gcc", *CFLAGS, "-fopenmp", SRC, "-o", LIB_OMP, "-lm"])
    procs = [subprocess.Popen(j, stdout=subprocess.PIPE, stderr=subprocess.STDOUT) for j in jobs]
    for j, p in zip(jobs, procs):
        out, _ = p.communicate()
        if verbose or p.returncode:
            sys.stderr.write(out.decode())
        if p.returncode:
            raise RuntimeError("oracle build failed: " + " ".join(j))
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
    print(LIB)
