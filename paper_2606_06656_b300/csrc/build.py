"""Build libcls_b300.so (sm_103a) in-tree with nvcc.

    python -m paper_2606_06656_b300.csrc.build [--force] [--verbose]

Objects go to paper_2606_06656_b300/_build/, the shared library to
paper_2606_06656_b300/libcls_b300.so.  Rebuilds only when a source or
header is newer than the library.
"""
import argparse
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
PKG = os.path.dirname(HERE)
ROOT = os.path.dirname(PKG)
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libcls_b300.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CUDA_SOURCES = ["kernels.cu", "kernels_p2.cu", "kernels_fr.cu", "kernels_corner.cu",
                "kernels_series.cu", "api.cu", "noalloc.cu", "mpnn.cu"]
CXX_SOURCES = ["plan.cpp"]


def nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources():
    out = [os.path.join(HERE, f) for f in os.listdir(HERE)
           if f.endswith((".cu", ".cuh", ".cpp", ".h"))]
    out += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return out


def needs_build():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources())


def _run(cmd, verbose):
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"build failed: {' '.join(cmd)}\n{r.stdout}")
    return r.stdout


def build(force=False, verbose=False, ptxas_verbose=False):
    if not force and not needs_build():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nv = nvcc()
    common = ["-O3", "-std=c++17", "-I", INCLUDE, "-Xcompiler", "-fPIC,-O3"]
    jobs = []
    for f in CUDA_SOURCES:
        obj = os.path.join(BUILD, f + ".o")
        extra = ["-Xptxas", "-v"] if ptxas_verbose else []
        jobs.append([nv, *ARCH, "-lineinfo", *common, *extra, "-c",
                     os.path.join(HERE, f), "-o", obj])
    for f in CXX_SOURCES:
        obj = os.path.join(BUILD, f + ".o")
        jobs.append([nv, *common, "-x", "c++", "-c", os.path.join(HERE, f), "-o", obj])
    logs = []
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        for out in ex.map(lambda c: _run(c, verbose), jobs):
            logs.append(out)
    objs = [os.path.join(BUILD, f + ".o") for f in CUDA_SOURCES + CXX_SOURCES]
    tmp = LIB + ".tmp"
    _run([nv, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"], verbose)
    os.replace(tmp, LIB)
    if ptxas_verbose:
        print("\n".join(logs))
    return LIB


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--verbose", action="store_true")
    ap.add_argument("--ptxas", action="store_true", help="print ptxas register/smem usage")
    a = ap.parse_args(argv)
    print(build(force=a.force, verbose=a.verbose, ptxas_verbose=a.ptxas))


if __name__ == "__main__":
    sys.exit(main())
