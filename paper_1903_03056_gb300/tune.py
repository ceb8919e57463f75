"""Autotuner of the collision kernel's launch shape and of its line transforms' radix schedule.

    python -m paper_1903_03056_gb300.tune [--precision fp32] [--sizes 16 24 32 48] [--write]
    python -m paper_1903_03056_gb300.tune --radix [--precision fp32] [--sizes 16 24 32 48] [--write]

For every grid size N it builds the kernel once per candidate shape -- thread-block cluster
size C, plane groups per CTA GP, CTAs per SM the registers are sized for (MB) -- in a
temporary copy of the sources (only the translation unit of that precision is recompiled and
linked with the current build's other objects), runs that build on the size's workload,
checks that its output is bitwise identical to the current build's (a shape changes which
thread computes a line, never the arithmetic of a line), and keeps the fastest.  With
--write the winners replace their lines of csrc/tuned_shapes.h and every timing is recorded
in csrc/tuned_shapes.json; rebuild afterwards.

With --radix it times, per N, every order of the radices 8, 4, 2, 3 in the candidate list
(tuned_radix.h codes) of the FP32 kernel instead.  A schedule changes the rounding of a line,
so its output is checked against the FP64 path on the first nodes of the workload (the largest
per-node max |Q - Q_fp64| / max |Q_fp64| must stay below the FP32 bar, 1e-5); the fastest
schedule that passes is kept.  (FP64 schedules stay at the default order: an FP64 variant has
no more accurate path to be checked against on the device.)
"""

import argparse
import json
import os
import re
import shutil
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

from . import build

PKG = build.PKG
ROOT = build.ROOT
CSRC = build.CSRC
SHAPES_H = os.path.join(CSRC, "tuned_shapes.h")
SHAPES_JSON = os.path.join(CSRC, "tuned_shapes.json")

WORKLOAD_FOR_N = {16: ("vhs_n16", 8192), 24: ("hs_n24", 16384), 32: ("dg_batch_n32", 4096),
                  48: ("vhs_n48", 512)}
CANDIDATES = {
    16: [(1, 8, 3), (1, 8, 1), (2, 4, 3), (1, 4, 4), (1, 16, 1)],
    24: [(2, 4, 3), (2, 12, 1), (1, 8, 2), (2, 4, 2)],
    32: [(2, 4, 1), (4, 4, 1), (1, 8, 1), (2, 8, 1), (2, 2, 2), (4, 2, 1), (8, 2, 1), (8, 4, 1),
         (4, 8, 1), (2, 2, 4), (4, 2, 4), (2, 1, 8), (1, 2, 4), (2, 4, 3), (1, 4, 3), (4, 4, 3),
         (2, 2, 6), (8, 4, 3), (4, 4, 2), (8, 4, 2), (8, 4, 4)],
    48: [(2, 4, 1), (2, 3, 1), (1, 4, 1), (2, 2, 2), (4, 4, 1), (4, 2, 1), (8, 2, 1)],
}


RADIX_H = os.path.join(CSRC, "tuned_radix.h")
# orders of the radix multisets of each N (4-stage and longer schedules left out)
RADIX_CANDIDATES = {
    12: [43, 34, 223, 232, 322],
    16: [44, 82, 28, 422, 242, 224],
    24: [423, 83, 38, 432, 243, 342, 234, 324],
    32: [442, 84, 48, 424, 244, 822, 282, 228],
    48: [443, 434, 344, 823, 832, 283, 238, 382, 328],
}
RADIX_BAR = 1e-5
RADIX_CHECK_NODES = 4


def radix_code_valid(N, code):
    """A schedule's radices are 2, 3, 4 or 8 and multiply to N."""
    digits = [int(c) for c in str(code)]
    prod = 1
    for d in digits:
        prod *= d
    return all(d in (2, 3, 4, 8) for d in digits) and prod == N


def _radix_line(T, N, code):
    return "DGFS_RADIX(%s, %d, %d)" % (T, N, code)


def _patch_radix(text, T, N, line):
    pat = re.compile(r"^DGFS_RADIX\(%s, %d, \d+\)$" % (T, N), re.M)
    if not pat.search(text):
        raise RuntimeError("no radix line for %s N=%d" % (T, N))
    return pat.sub(line, text)


def geometry(N, C, GP, MB, csize):
    """The kernel's compile-time geometry of a shape (the same rules as its Geo template):
    P in registers, CTAs per SM, y-pass sharing, tensor-memory accumulators, plane buffers per
    group and the shared memory of the plane buffers.  csize = bytes of one complex element."""
    preg = (csize == 8 and N <= 48) or N <= 16
    buf = N * (N + 1) * csize
    threads = GP * N
    if MB > 1:
        res = MB
    else:
        res = 2 if threads <= 128 and 2 * (GP * 2 * buf + 1024) <= 228 * 1024 else 1
    ysh = N <= 16 and preg and res * (GP * 3 * buf + 1024 + 8 * 1024) <= 228 * 1024
    # tensor-memory accumulators: P of the group's planes and a_e in 2N FP32 columns per line
    ppg = (N // C) // GP
    tm_cols = 2 * N * (ppg + 1)
    tm_alloc = next(a for a in (32, 64, 128, 256, 512, 1 << 30) if tm_cols <= a)
    tm = csize == 8 and N % 32 == 0 and threads <= 128 and not ysh and tm_cols <= 512 and res * tm_alloc <= 512
    nbuf = 1 if tm else 2 if preg and not ysh else 3
    return {"preg": preg, "res": res, "ysh": ysh, "tm": tm, "nbuf": nbuf, "threads": threads,
            "smem": GP * nbuf * buf}


def valid(N, C, GP, MB, csize):
    """Shape constraints of the kernel: planes and pencils split evenly over the cluster and
    the plane groups, at most 1024 threads, the plane buffers of MB CTAs in one SM's shared
    memory, and at least 64 registers a thread at MB CTAs per SM."""
    if N % C or (N * N) % C or (N // C) % GP or GP * N > 1024:
        return False
    g = geometry(N, C, GP, MB, csize)
    return MB * g["smem"] <= 227 * 1024 and 65536 // (g["threads"] * MB) >= 64


def _ctype(precision):
    return "float" if precision == "fp32" else "double"


def _shape_line(T, N, C, GP, MB):
    return "DGFS_SHAPE3(%s, %d, %d, %d, %d)" % (T, N, C, GP, MB)


def _patch(text, T, N, line):
    pat = re.compile(r"^DGFS_SHAPE3?\(%s, %d,[^\n]*\)$" % (T, N), re.M)
    if not pat.search(text):
        raise RuntimeError("no shape line for %s N=%d" % (T, N))
    return pat.sub(line, text)


def _variant(tmp, precision, N, shape, radix=None):
    """Build a variant tree under tmp; returns its root (with the package inside).  With
    `radix` the shape stays and the radix schedule of (precision, N) becomes `radix`."""
    T = _ctype(precision)
    C, GP, MB = shape
    root = os.path.join(tmp, "%s_%d_%d_%d_%d_r%s" % (precision, N, C, GP, MB, radix))
    pkg = os.path.join(root, "paper_1903_03056_gb300")
    os.makedirs(os.path.join(pkg, "_build"))
    for f in os.listdir(PKG):
        if f.endswith(".py"):
            shutil.copy(os.path.join(PKG, f), pkg)
    shutil.copytree(CSRC, os.path.join(pkg, "csrc"))
    shutil.copytree(os.path.join(ROOT, "include"), os.path.join(root, "include"))
    h = os.path.join(pkg, "csrc", "tuned_shapes.h")
    with open(h) as fh:
        text = fh.read()
    with open(h, "w") as fh:
        fh.write(_patch(text, T, N, _shape_line(T, N, C, GP, MB)))
    if radix is not None:
        rh = os.path.join(pkg, "csrc", "tuned_radix.h")
        with open(rh) as fh:
            text = fh.read()
        with open(rh, "w") as fh:
            fh.write(_patch_radix(text, T, N, _radix_line(T, N, radix)))
    tu = "collision_f32" if precision == "fp32" else "collision_f64"
    obj = os.path.join(pkg, "_build", tu + ".o")
    cmd = ([build.nvcc()] + build.ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
           "-I" + os.path.join(root, "include"), "-I" + os.path.join(pkg, "csrc"), "-c",
           os.path.join(pkg, "csrc", tu + ".cu"), "-o", obj])
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(res.stderr[-2000:])
    others = [os.path.join(build.BUILD, f) for f in os.listdir(build.BUILD)
              if f.endswith(".o") and f != tu + ".o"]
    res = subprocess.run([build.nvcc()] + build.ARCH + ["-shared", "-o", os.path.join(pkg, "libdgfs.so"), obj] + others,
                         capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(res.stderr[-2000:])
    os.utime(os.path.join(pkg, "libdgfs.so"))
    return root


def _time(root, workload, batch, precision, compare=0):
    env = dict(os.environ, PYTHONPATH=root + os.pathsep + ROOT)
    extra = ["--compare-fp64", str(compare)] if compare else []
    res = subprocess.run([sys.executable, "-m", "paper_1903_03056_gb300.run_case", "--workload", workload,
                          "--batch", str(batch), "--precision", precision, "--repeat", "3", "--checksum"] + extra,
                         capture_output=True, text=True, cwd=root, env=env)
    if res.returncode != 0:
        raise RuntimeError(res.stderr[-2000:])
    return json.loads(res.stdout.strip().splitlines()[-1])


def tune(precision="fp32", sizes=(16, 24, 32, 48), write=False, jobs=8):
    build.build()
    csize = 8 if precision == "fp32" else 16
    T = _ctype(precision)
    record = {}
    if os.path.exists(SHAPES_JSON):
        with open(SHAPES_JSON) as fh:
            record = json.load(fh)
    with open(SHAPES_H) as fh:
        header = fh.read()
    with tempfile.TemporaryDirectory(prefix="dgfs_tune_") as tmp:
        todo = [(N, sh) for N in sizes for sh in CANDIDATES.get(N, []) if valid(N, *sh, csize)]
        with ThreadPoolExecutor(max_workers=jobs) as ex:
            roots = dict(zip(todo, ex.map(lambda t: _variant(tmp, precision, t[0], t[1]), todo)))
        for N in sizes:
            workload, batch = WORKLOAD_FOR_N[N]
            ref = _time(ROOT, workload, batch, precision)
            rows = []
            for sh in CANDIDATES.get(N, []):
                if (N, sh) not in roots:
                    continue
                r = _time(roots[(N, sh)], workload, batch, precision)
                rows.append({"cluster": sh[0], "groups": sh[1], "ctas_per_sm": sh[2], "ms": r["ms"],
                             "identical": r["sha1"] == ref["sha1"]})
                print("%s N=%d C=%d GP=%d MB=%d: %.2f ms%s" % (precision, N, sh[0], sh[1], sh[2], r["ms"],
                      "" if rows[-1]["identical"] else "  (output differs: rejected)"), flush=True)
            ok = [r for r in rows if r["identical"]]
            if not ok:
                continue
            best = min(ok, key=lambda r: r["ms"])
            record["%s/%d" % (precision, N)] = {"workload": workload, "batch": batch, "current_ms": ref["ms"],
                                               "best": best, "candidates": rows}
            header = _patch(header, T, N, _shape_line(T, N, best["cluster"], best["groups"], best["ctas_per_sm"]))
    if write:
        with open(SHAPES_H, "w") as fh:
            fh.write(header)
        with open(SHAPES_JSON, "w") as fh:
            json.dump(record, fh, indent=1, sort_keys=True)
    return record


def current_shape(precision, N):
    """(cluster, groups, CTAs per SM) of (precision, N) in tuned_shapes.h."""
    T = _ctype(precision)
    with open(SHAPES_H) as fh:
        text = fh.read()
    m = re.search(r"^DGFS_SHAPE(3?)\(%s, %d, (\d+), (\d+)(?:, (\d+))?\)$" % (T, N), text, re.M)
    return int(m.group(2)), int(m.group(3)), int(m.group(4) or 1)


def current_radix(precision, N):
    with open(RADIX_H) as fh:
        m = re.search(r"^DGFS_RADIX\(%s, %d, (\d+)\)$" % (_ctype(precision), N), fh.read(), re.M)
    return int(m.group(1))


def tune_radix(precision="fp32", sizes=(16, 24, 32, 48), write=False, jobs=8):
    """Time every candidate radix schedule of each N at the current launch shape; keep the fastest
    whose output stays within RADIX_BAR of the FP64 path."""
    if precision != "fp32":
        raise ValueError("radix schedules are tuned for the FP32 kernel")
    build.build()
    T = _ctype(precision)
    record = {}
    if os.path.exists(SHAPES_JSON):
        with open(SHAPES_JSON) as fh:
            record = json.load(fh)
    with open(RADIX_H) as fh:
        header = fh.read()
    with tempfile.TemporaryDirectory(prefix="dgfs_tune_") as tmp:
        todo = [(N, code) for N in sizes for code in RADIX_CANDIDATES.get(N, []) if radix_code_valid(N, code)]
        with ThreadPoolExecutor(max_workers=jobs) as ex:
            roots = dict(zip(todo, ex.map(lambda t: _variant(tmp, precision, t[0], current_shape(precision, t[0]),
                                                             radix=t[1]), todo)))
        for N in sizes:
            workload, batch = WORKLOAD_FOR_N[N]
            cur = current_radix(precision, N)
            rows = []
            for code in RADIX_CANDIDATES.get(N, []):
                if (N, code) not in roots:
                    continue
                r = _time(roots[(N, code)], workload, batch, precision, compare=RADIX_CHECK_NODES)
                ok = r["err_vs_fp64"] < RADIX_BAR
                rows.append({"radix": code, "ms": r["ms"], "err_vs_fp64": r["err_vs_fp64"], "ok": ok})
                print("%s N=%d radix %d: %.2f ms, error vs FP64 %.2e%s" % (precision, N, code, r["ms"], r["err_vs_fp64"],
                      "" if ok else "  (above the bar: rejected)"), flush=True)
            good = [r for r in rows if r["ok"]]
            if not good:
                continue
            best = min(good, key=lambda r: r["ms"])
            record["radix/%s/%d" % (precision, N)] = {"workload": workload, "batch": batch, "previous": cur,
                                                     "shape": list(current_shape(precision, N)), "best": best,
                                                     "candidates": rows}
            header = _patch_radix(header, T, N, _radix_line(T, N, best["radix"]))
    if write:
        with open(RADIX_H, "w") as fh:
            fh.write(header)
        with open(SHAPES_JSON, "w") as fh:
            json.dump(record, fh, indent=1, sort_keys=True)
    return record


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--sizes", type=int, nargs="+", default=[16, 24, 32, 48])
    ap.add_argument("--write", action="store_true")
    ap.add_argument("--jobs", type=int, default=8)
    ap.add_argument("--radix", action="store_true", help="tune the radix schedules instead of the launch shapes")
    a = ap.parse_args()
    if a.radix:
        rec = tune_radix(a.precision, tuple(a.sizes), a.write, a.jobs)
    else:
        rec = tune(a.precision, tuple(a.sizes), a.write, a.jobs)
    print(json.dumps({k: v["best"] for k, v in rec.items()}, indent=1))
