"""Build the in-tree CUDA library libdgmax.so for sm_103a (GB300).

Every translation unit under csrc/ is compiled by nvcc in parallel and linked
into paper_2002_08733_gb300/_lib/libdgmax.so.  Objects are rebuilt when their
source or any header changed.
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
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
GEN = os.path.join(BUILD, "gen")
GEN_HEADER = os.path.join(GEN, "dgm_ops_gen.cuh")
GENERATOR_SRC = ("dgm_refgen.cpp", "dgm_refmats.cpp")
LIBDIR = os.path.join(PKG, "_lib")
LIB = os.path.join(LIBDIR, "libdgmax.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC, "-I", GEN]


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found")
    return exe


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC)
                  if (f.endswith(".cu") or f.endswith(".cpp")) and f != "dgm_refgen.cpp")


def headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hs += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    if os.path.exists(GEN_HEADER):
        hs.append(GEN_HEADER)
    return hs


def generate_operators():
    """Compile and run dgm_refgen (host) to write the straight-line reference operators."""
    os.makedirs(GEN, exist_ok=True)
    srcs = [os.path.join(CSRC, f) for f in GENERATOR_SRC]
    deps = srcs + [os.path.join(CSRC, "dgm_internal.h")]
    newest = max(os.path.getmtime(d) for d in deps)
    if os.path.exists(GEN_HEADER) and os.path.getmtime(GEN_HEADER) >= newest:
        return
    exe = os.path.join(BUILD, "refgen")
    cmd = [nvcc(), "-x", "c++", "-O2", "-std=c++17", "-I", INCLUDE, "-I", CSRC] + srcs + ["-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("generator build failed:\n%s\n%s" % (r.stdout, r.stderr))
    tmp = GEN_HEADER + ".tmp"
    r = subprocess.run([exe, tmp], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("generator failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, GEN_HEADER)


def _compile(src, extra):
    obj = os.path.join(BUILD, os.path.basename(src) + ".o")
    newest_dep = max([os.path.getmtime(src)] + [os.path.getmtime(h) for h in headers()])
    if os.path.exists(obj) and os.path.getmtime(obj) >= newest_dep:
        return obj, None
    lang = ["-x", "cu"] if src.endswith(".cu") else ["-x", "c++"]
    cmd = [nvcc()] + ARCH + FLAGS + extra + lang + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        return obj, "%s\n%s\n%s" % (" ".join(cmd), r.stdout, r.stderr)
    return obj, None


def build(verbose=False, jobs=None, extra=()):
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    generate_operators()
    srcs = sources()
    jobs = jobs or min(len(srcs), os.cpu_count() or 4)
    errors, objs = [], []
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        for obj, err in ex.map(lambda s: _compile(s, list(extra)), srcs):
            objs.append(obj)
            if err:
                errors.append(err)
    if errors:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
    newest = max(os.path.getmtime(o) for o in objs)
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < newest:
        cmd = [nvcc()] + ARCH + ["-shared", "-o", LIB] + objs + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build(verbose=True, extra=sys.argv[1:])
