"""Build the CUDA library libgbsz.so in-tree for sm_103a (GB300).

Each translation unit compiles in parallel with nvcc; the shared library
links the CUDA runtime statically.  Objects go to _build/ at the repo root.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libgbsz.so")
# the bounds-checking build: every GBSZ_CHECK in the kernels compiled in
CHECK_BUILD = os.path.join(ROOT, "_build_check")
CHECK_LIB = os.path.join(PKG, "libgbsz_check.so")
SOURCES = ["gbsz_api.cu", "k_quant.cu", "k_codebook.cu", "k_encode.cu", "k_decode.cu", "k_decode_warp.cu", "k_recon.cu",
           "noalloc.cu", "server.cu"]
HEADERS = ["common.cuh", "scan.cuh", "server_core.h"]

NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -fmad=false: no contraction of the few float multiplies and adds, whose
# rounding the archive format fixes (each is one IEEE round-to-nearest op).
FLAGS = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-fmad=false", "-Xcompiler", "-fPIC",
                "-I" + os.path.join(ROOT, "include")]


def _newest_input():
    paths = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    paths.append(os.path.join(ROOT, "include", "gbsz.h"))
    paths.append(os.path.abspath(__file__))
    return max(os.path.getmtime(p) for p in paths)


def build(force=False, verbose=False, extra_flags=(), check=False):
    """check=True: the bounds-checking build (-DGBSZ_BOUNDS_CHECK) into
    libgbsz_check.so, objects in _build_check/."""
    lib, bdir = (CHECK_LIB, CHECK_BUILD) if check else (LIB, BUILD)
    if check:
        extra_flags = tuple(extra_flags) + ("-DGBSZ_BOUNDS_CHECK",)
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _newest_input():
        return lib
    os.makedirs(bdir, exist_ok=True)

    def compile_one(src):
        obj = os.path.join(bdir, src.replace(".cu", ".o"))
        cmd = [NVCC, *FLAGS, *extra_flags, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
        return src, obj, r.returncode, r.stdout.decode()

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    failed = [r for r in results if r[2] != 0]
    for src, _, rc, out in results:
        if verbose or rc:
            sys.stderr.write(out)
    if failed:
        raise RuntimeError("nvcc failed for " + ", ".join(r[0] for r in failed))
    objs = [r[1] for r in results]
    tmp = lib + ".tmp"
    cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode:
        sys.stderr.write(r.stdout.decode())
        raise RuntimeError("link failed")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
