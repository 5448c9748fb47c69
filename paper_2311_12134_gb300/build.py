"""Build liblsmskubo.so in-tree for sm_103a (nvcc + g++, no cmake).

    python -m paper_2311_12134_gb300.build

Compiles the CUDA translation units and the host C++ file in parallel and links
them into ``paper_2311_12134_gb300/_lib/liblsmskubo.so``.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liblsmskubo.so")

CUDA_SOURCES = ["api.cu", "lu.cu", "kubo.cu", "tc_gemm.cu", "resid_tc.cu"]
CXX_SOURCES = ["host.cpp"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _cuda_home():
    for cand in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "bin", "nvcc")):
            return cand
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("nvcc not found; set CUDA_HOME")


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("command failed:\n" + " ".join(cmd) + "\n" + r.stdout)
    return r.stdout


def build(verbose=False, extra_nvcc=()):
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    os.makedirs(OUT_DIR, exist_ok=True)
    os.makedirs(BUILD_DIR, exist_ok=True)
    inc = ["-I" + os.path.join(HERE, "..", "include"), "-I" + CSRC]
    jobs = []
    for src in CUDA_SOURCES:
        obj = os.path.join(BUILD_DIR, src + ".o")
        jobs.append([nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-Xptxas", "-v" if verbose else "-O3", *extra_nvcc, *inc, "-c",
                     os.path.join(CSRC, src), "-o", obj])
    for src in CXX_SOURCES:
        obj = os.path.join(BUILD_DIR, src + ".o")
        jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-pthread", "-ffp-contract=off", *inc, "-c",
                     os.path.join(CSRC, src), "-o", obj])
    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        outs = list(ex.map(_run, jobs))
    if verbose:
        for o in outs:
            sys.stdout.write(o)
    objs = [os.path.join(BUILD_DIR, s + ".o") for s in CUDA_SOURCES + CXX_SOURCES]
    tmp = LIB + ".tmp"
    _run([nvcc, ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs, "-lpthread",
          "-Xlinker", "-rpath=" + os.path.join(cuda, "lib64")])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
