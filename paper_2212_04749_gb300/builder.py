"""Build the contraction library in-tree: ``paper_2212_04749_gb300/_lib/libtn.so``.

nvcc compiles each CUDA translation unit for sm_103a only
(``-gencode arch=compute_103a,code=sm_103a``) and g++ the host planner; the
units build in parallel and are linked into one shared library against the
CUDA runtime.  Nothing here is machine specific (no -march flags), so the
same command builds on x86_64 and aarch64 hosts.
"""

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libtn.so")
ROOT = os.path.dirname(HERE)

CU_SOURCES = ["kernels.cu", "gemm_tc.cu", "chain.cu", "mlp.cu", "api.cu"]
CPP_SOURCES = ["plan.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    cand = os.path.join(cuda, "bin", "nvcc")
    return cand if os.path.exists(cand) else (shutil.which("nvcc") or "nvcc")


def _sources():
    return [os.path.join(CSRC, f) for f in CU_SOURCES + CPP_SOURCES] + [
        os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".hpp"))
    ] + [os.path.join(ROOT, "include", "tn.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    objdir = os.path.join(OUT_DIR, "obj")
    os.makedirs(objdir, exist_ok=True)
    nvcc = _nvcc()
    inc = ["-I", os.path.join(ROOT, "include")]
    cmds = []
    objs = []
    for f in CU_SOURCES:
        o = os.path.join(objdir, f + ".o")
        objs.append(o)
        cmds.append([nvcc, "-std=c++17", "-O3", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
                     "-Xptxas", "-v" if verbose else "-O3", *inc, "-c", os.path.join(CSRC, f), "-o", o])
    for f in CPP_SOURCES:
        o = os.path.join(objdir, f + ".o")
        objs.append(o)
        cmds.append(["g++", "-std=c++17", "-O2", "-fPIC", *inc, "-c", os.path.join(CSRC, f), "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    with ThreadPoolExecutor(max_workers=len(cmds)) as ex:
        for cmd, r in ex.map(run, cmds):
            if verbose and (r.stdout or r.stderr):
                sys.stderr.write(r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError("build failed: " + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    tmp = LIB + ".tmp"
    link = [nvcc, "-shared", *ARCH, "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed: " + " ".join(link) + "\n" + r.stdout + r.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
