"""Build the CUDA library ``libfrgb.so`` in-tree for sm_103a.

Host C++ translation units are compiled with g++, CUDA units with nvcc for
``-gencode arch=compute_103a,code=sm_103a`` only, in parallel, then linked
into ``paper_2408_16509_gb300/lib/libfrgb.so``.  Rebuilds only when a source
is newer than the library.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OUT_DIR = os.path.join(HERE, "lib")
OBJ_DIR = os.path.join(HERE, "lib", "obj")
LIB = os.path.join(OUT_DIR, "libfrgb.so")

ARCH = "-gencode=arch=compute_103a,code=sm_103a"
CXX_SRCS = ["fr_ref.cpp", "fr_mesh.cpp", "fr_part.cpp"]
CU_SRCS = ["fr_api.cu", "fr_prec_f64.cu", "fr_prec_f32.cu", "fr_prec_mix.cu", "fr_probe.cu"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc",
                 shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required")


def _sources():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)
             if f.endswith((".cu", ".cuh", ".cpp", ".hpp"))]
    files.append(os.path.join(INCLUDE, "frgb.h"))
    files.append(os.path.abspath(__file__))
    return files


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in _sources())


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n"
                           + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(force=False, verbose=False, ptxas_info=False):
    """Compile the library if needed and return the path of the .so."""
    if not force and not _stale():
        return LIB
    os.makedirs(OBJ_DIR, exist_ok=True)
    nvcc = _nvcc()
    jobs = []
    for src in CXX_SRCS:
        obj = os.path.join(OBJ_DIR, src + ".o")
        jobs.append([shutil.which("g++") or "g++", "-std=c++17", "-O2",
                     "-fPIC", "-pthread", "-c", os.path.join(CSRC, src), "-o", obj,
                     "-I" + INCLUDE])
    for src in CU_SRCS:
        obj = os.path.join(OBJ_DIR, src + ".o")
        cmd = [nvcc, "-std=c++17", "-O3", ARCH, "-lineinfo",
               "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
               "-c", os.path.join(CSRC, src), "-o", obj, "-I" + INCLUDE]
        if ptxas_info:
            cmd.insert(1, "-Xptxas=-v")
        jobs.append(cmd)
    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        logs = list(ex.map(_run, jobs))
    if verbose:
        for lg in logs:
            sys.stdout.write(lg)
    objs = [os.path.join(OBJ_DIR, s + ".o") for s in CXX_SRCS + CU_SRCS]
    _run([nvcc, "-shared", ARCH, "-o", LIB] + objs + ["-lcudart", "-lpthread"])
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          ptxas_info="--ptxas" in sys.argv)
    print(LIB)
