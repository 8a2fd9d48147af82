"""Build the CUDA shared library in place (nvcc, sm_103a only).

Each translation unit under csrc/ is compiled in parallel into _build/, then
linked into libgb300stencil.so next to this file. Rebuilds only what changed.
The checked build (the same sources with -DSTENCIL_CHECKED: every kernel index
tested before its access, see stencil_checked_build in include/stencil.h) goes
to _build/checked/ and libgb300stencil_checked.so. The FP64 pipe
micro-benchmark (peak/fp64_peak.cu, the ALU roofline bench.py reports against)
is compiled alongside into peak/fp64_peak.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libgb300stencil.so")
LIB_CHECKED = os.path.join(HERE, "libgb300stencil_checked.so")
SOURCES = ["abi.cu", "k_plain.cu", "k_blocked.cu", "k_stream.cu", "k_diamond.cu", "k_wavefront.cu", "tune.cu", "k_noalloc.cu", "k_batch.cu", "k_life.cu", "k_lcs.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
         "-Xcompiler", "-fno-strict-aliasing", "-I", os.path.join(ROOT, "include")]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _deps():
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    inc = os.path.join(ROOT, "include")
    hdrs += [os.path.join(inc, f) for f in os.listdir(inc) if f.endswith(".h")]
    return max(os.path.getmtime(h) for h in hdrs)


def _compile(src, hdr_mtime, extra, outdir=BUILD):
    obj = os.path.join(outdir, src.replace(".cu", ".o"))
    s = os.path.join(CSRC, src)
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(s), hdr_mtime):
        return obj, None
    cmd = [_nvcc()] + ARCH + FLAGS + extra + ["-c", s, "-o", obj]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        return obj, "%s\n%s%s" % (" ".join(cmd), p.stdout, p.stderr)
    return obj, None


PROBE_SRC = os.path.join(HERE, "peak", "fp64_peak.cu")
PROBE_EXE = os.path.join(HERE, "peak", "fp64_peak")


def build_probe() -> str:
    """Compile the FP64 pipe micro-benchmark into peak/fp64_peak (if its source is newer)."""
    if os.path.exists(PROBE_EXE) and os.path.getmtime(PROBE_EXE) >= os.path.getmtime(PROBE_SRC):
        return PROBE_EXE
    tmp = PROBE_EXE + ".tmp%d" % os.getpid()
    cmd = [_nvcc()] + ARCH + ["-O3", "-o", tmp, PROBE_SRC]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError("nvcc failed:\n%s\n%s%s" % (" ".join(cmd), p.stdout, p.stderr))
    os.replace(tmp, PROBE_EXE)
    return PROBE_EXE


def _link(objs, lib):
    if not os.path.exists(lib) or os.path.getmtime(lib) < max(os.path.getmtime(o) for o in objs):
        tmp = lib + ".tmp%d" % os.getpid()
        cmd = [_nvcc()] + ARCH + ["-shared", "-o", tmp] + objs
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s%s" % (" ".join(cmd), p.stdout, p.stderr))
        os.replace(tmp, lib)


def build(verbose: bool = False, extra=(), checked: bool = True) -> str:
    """Compile and link the library (and, unless checked=False, its checked build, in the same pool)."""
    variants = [(BUILD, LIB, list(extra))]
    if checked:
        variants.append((os.path.join(BUILD, "checked"), LIB_CHECKED, list(extra) + ["-DSTENCIL_CHECKED"]))
    for d, _, _ in variants:
        os.makedirs(d, exist_ok=True)
    hdr = _deps()
    jobs = [(s, d, x) for d, _, x in variants for s in SOURCES]
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        probe = ex.submit(build_probe)
        res = list(ex.map(lambda j: _compile(j[0], hdr, j[2], j[1]), jobs))
        probe.result()
    errs = [e for _, e in res if e]
    if errs:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errs))
    for k, (_, lib, _) in enumerate(variants):
        _link([o for o, _ in res[k * len(SOURCES):(k + 1) * len(SOURCES)]], lib)
        if verbose:
            print(lib)
    return LIB


if __name__ == "__main__":
    build(verbose=True, extra=sys.argv[1:])
