"""Build libdgfs.so in-tree with nvcc for sm_103a (GB300).

    python -m paper_1903_03056_gb300.build [--force] [--verbose]

Translation units compile in parallel; the library is rebuilt when the SHA-1 of its sources,
headers and build flags differs from the one recorded at its last build (or the library is
missing).  ptxas resource usage (registers, spills, shared memory) is written to
``_build/ptxas.log`` beside the objects.
"""

import argparse
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libdgfs.so")

SOURCES = ["api.cpp", "plan.cpp", "collision_f32.cu", "collision_f64.cu", "collision_noalloc.cu", "conserve.cu", "tables.cu",
           "stepper.cu", "dg1d.cu", "peaks.cu", "dft_gemm.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]


def nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "dgfs.h"))
    files.append(os.path.abspath(__file__))
    return files


STAMP = os.path.join(BUILD, "sources.sha1")


def sources_sha1():
    """SHA-1 over every source and header of the library and the compile flags."""
    import hashlib
    h = hashlib.sha1(" ".join(ARCH + FLAGS + SOURCES).encode())
    for f in sorted(_deps()):
        with open(f, "rb") as fh:
            h.update(os.path.basename(f).encode() + b"\0" + fh.read())
    return h.hexdigest()


def up_to_date():
    if not os.path.exists(LIB) or not os.path.exists(STAMP):
        return False
    with open(STAMP) as fh:
        return fh.read().strip() == sources_sha1()


def _compile(src):
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc()] + ARCH + FLAGS + ["-c", os.path.join(CSRC, src), "-o", obj]
    if src.endswith(".cu"):
        cmd += ["-Xptxas", "-v"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    return src, obj, res


def build(force=False, verbose=False):
    """Compile every translation unit and link libdgfs.so; returns the library path."""
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(_compile, SOURCES))
    log = []
    for src, obj, res in results:
        log.append("== %s\n%s%s" % (src, res.stdout, res.stderr))
        if res.returncode != 0:
            sys.stderr.write(res.stdout + res.stderr)
            raise RuntimeError("nvcc failed on %s" % src)
    with open(os.path.join(BUILD, "ptxas.log"), "w") as fh:
        fh.write("\n".join(log))
    objs = [obj for _, obj, _ in results]
    tmp = LIB + ".tmp"
    res = subprocess.run([nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-ldl"], capture_output=True, text=True)
    if res.returncode != 0:
        sys.stderr.write(res.stdout + res.stderr)
        raise RuntimeError("link failed")
    os.replace(tmp, LIB)
    with open(STAMP, "w") as fh:
        fh.write(sources_sha1() + "\n")
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--verbose", action="store_true")
    a = ap.parse_args()
    build(force=a.force, verbose=True)
