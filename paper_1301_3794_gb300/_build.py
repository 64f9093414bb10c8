"""Build libdmeig.so in-tree with nvcc for sm_103a (GB300).

Every translation unit is compiled in parallel, then linked into
``paper_1301_3794_gb300/libdmeig.so``.  Objects go to ``paper_1301_3794_gb300/_build``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libdmeig.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
          "--expt-relaxed-constexpr"]
# per-file extra flags: the geometry is compiled without FMA contraction so that
# fraction sums (and the 0 < V < 1 band tests) round identically on every build
EXTRA = {"dm_geometry.cu": ["-fmad=false"]}
SOURCES = ["dm_geometry.cu", "dm_stencil.cu", "dm_band.cu", "dm_transfer.cu", "dm_blas.cu", "dm_dense.cu", "dm_learned.cu", "dm_conv_tc.cu", "dm_probe.cu",
           "dm_api.cu"]


def nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdmeig")


def _stale(obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose=False, force=False, jobs=None):
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    headers = [os.path.join(CSRC, "dm_common.cuh"), os.path.join(CSRC, "dm_learned.cuh"), os.path.join(INCLUDE, "dmeig.h")]
    cmds = []
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + headers):
            cmds.append([cc, *ARCH, *COMMON, *EXTRA.get(src, []), "-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, file=sys.stderr)
        return cmd[-1]

    with cf.ThreadPoolExecutor(max_workers=jobs or min(len(cmds) or 1, os.cpu_count() or 4)) as ex:
        list(ex.map(run, cmds))
    if force or cmds or _stale(LIB, objs):
        link = [cc, *ARCH, "-shared", "-o", LIB, *objs]
        run(link)
    return LIB


if __name__ == "__main__":
    build(verbose=True, force="--force" in sys.argv)
    print(LIB)
