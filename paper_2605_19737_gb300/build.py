"""Compile the CUDA library libvr.so in-tree for sm_103a (GB300).

Each translation unit under csrc/ is compiled in parallel with nvcc
(-gencode arch=compute_103a,code=sm_103a -O3 -lineinfo) and linked into
paper_2605_19737_gb300/libvr.so; the same sources with -DVR_DEBUG (kernel index
checks that report through the context's status word) give libvr_debug.so.
Nothing here needs a GPU.
"""

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT = os.path.join(PKG, "libvr.so")
OUT_DEBUG = os.path.join(PKG, "libvr_debug.so")
BUILD = os.path.join(PKG, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# Host code is built without floating-point contraction so that host-side arithmetic
# (NIfTI intensity scaling) rounds the same way on x86-64 and aarch64 hosts.
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
         "-I" + INCLUDE, "-I" + CSRC]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libvr.so")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False, debug=None):
    """Build libvr.so (debug=False), libvr_debug.so (debug=True) or both (None, the
    default), recompiling only translation units whose source or headers changed.
    Returns the path of libvr.so (of libvr_debug.so when debug=True)."""
    nvcc = _nvcc()
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    variants = {False: [False], True: [True], None: [False, True]}[debug]
    links, jobs = [], []
    for dbg in variants:
        bdir = os.path.join(BUILD, "debug") if dbg else BUILD
        os.makedirs(bdir, exist_ok=True)
        objs = []
        for src in sources():
            obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
            objs.append(obj)
            if force or _stale(obj, [src] + headers):
                jobs.append([nvcc] + ARCH + FLAGS + (["-DVR_DEBUG"] if dbg else []) + ["-c", src, "-o", obj])
        links.append((OUT_DEBUG if dbg else OUT, objs))

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n%s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            list(ex.map(run, jobs))
    for out, objs in links:
        if force or jobs or _stale(out, objs):
            tmp = out + ".tmp%d" % os.getpid()
            run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs)
            os.replace(tmp, out)
    return OUT_DEBUG if debug else OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
