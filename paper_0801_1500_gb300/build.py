"""Build ``libgbrt.so`` (the CUDA library behind include/gbrt.h) in-tree.

Each translation unit is compiled by nvcc for sm_103a in parallel, then linked
into one shared library next to this file. No cmake; a rebuild happens when a
source or header is newer than the library.

Beside it, ``libgbrt_checked.so``: the same library with the render kernels
and the C ABI compiled with -DGBRT_CHECKED, so every index that comes from
data is tested against its buffer (an index outside it is counted, replaced
by 0, and reported by gbrt_sync as GBRT_EBOUNDS). The binding loads it when
GBRT_LIB_VARIANT=checked; the tests use it to show that no workload reads or
writes outside a buffer.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libgbrt.so")
LIB_CHECKED = os.path.join(PKG, "libgbrt_checked.so")
# translation units whose code differs in the checked build
CHECKED_UNITS = ("render.cu", "capi.cu")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        [os.path.join(INCLUDE, "gbrt.h"), os.path.abspath(__file__)]


def up_to_date() -> bool:
    if not (os.path.exists(LIB) and os.path.exists(LIB_CHECKED)):
        return False
    t = min(os.path.getmtime(LIB), os.path.getmtime(LIB_CHECKED))
    return all(os.path.getmtime(p) <= t for p in _deps())


def cflags(ptxas_verbose: bool = False):
    f = ["-O3", "-std=c++17", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC,-fvisibility=hidden",
         "-I", INCLUDE, "-I", CSRC]
    if ptxas_verbose:
        f += ["-Xptxas", "-v"]
    return f


def _link(cc, objs, out):
    tmp = out + ".tmp"
    r = subprocess.run([cc, "-shared", *ARCH, "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stderr)
    os.replace(tmp, out)


def build(force: bool = False, verbose: bool = False, ptxas_verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(os.path.join(BUILD, "checked"), exist_ok=True)
    cc = nvcc()
    # every unit once, and the checked build's units again with -DGBRT_CHECKED,
    # all in one pool
    jobs = [(src, False) for src in _sources()] + \
        [(src, True) for src in _sources() if os.path.basename(src) in CHECKED_UNITS]

    def compile_one(job):
        src, checked = job
        obj = os.path.join(BUILD, "checked" if checked else "", os.path.basename(src)[:-3] + ".o")
        cmd = [cc, *cflags(ptxas_verbose), *(["-DGBRT_CHECKED"] if checked else []), "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        return src, checked, obj, r, cmd

    objs, checked_objs = {}, {}
    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        for src, checked, obj, r, cmd in ex.map(compile_one, jobs):
            if verbose or ptxas_verbose:
                print(" ".join(cmd))
                sys.stdout.write(r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {os.path.basename(src)}{' (checked)' if checked else ''}:\n"
                                   f"{r.stderr}")
            (checked_objs if checked else objs)[os.path.basename(src)] = obj
    _link(cc, [objs[k] for k in sorted(objs)], LIB)
    _link(cc, [checked_objs.get(k, objs[k]) for k in sorted(objs)], LIB_CHECKED)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, ptxas_verbose="--ptxas" in sys.argv))
