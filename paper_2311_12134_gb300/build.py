"""Build liblsmskubo.so in-tree for sm_103a (nvcc + g++, no cmake).

    python -m paper_2311_12134_gb300.build [--debug-bounds]

Compiles the CUDA translation units and the host C++ file in parallel and links
them into ``paper_2311_12134_gb300/_lib/liblsmskubo.so``.  ``--debug-bounds``
builds ``liblsmskubo_debug.so`` with -DLSMS_DEBUG_BOUNDS (device-side index
checks that flag a unit LSMS_UNIT_BAD_INPUT instead of accessing out of range);
the binding loads it when the environment sets LSMS_DEBUG_BOUNDS=1.
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
LIB_DEBUG = os.path.join(OUT_DIR, "liblsmskubo_debug.so")

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


def build(verbose=False, extra_nvcc=(), debug_bounds=False):
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    build_dir = BUILD_DIR + ("_debug" if debug_bounds else "")
    lib_path = LIB_DEBUG if debug_bounds else LIB
    if debug_bounds:
        extra_nvcc = (*extra_nvcc, "-DLSMS_DEBUG_BOUNDS")
    os.makedirs(OUT_DIR, exist_ok=True)
    os.makedirs(build_dir, exist_ok=True)
    inc = ["-I" + os.path.join(HERE, "..", "include"), "-I" + CSRC]
    jobs = []
    for src in CUDA_SOURCES:
        obj = os.path.join(build_dir, src + ".o")
        jobs.append([nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-Xptxas", "-v" if verbose else "-O3", *extra_nvcc, *inc, "-c",
                     os.path.join(CSRC, src), "-o", obj])
    for src in CXX_SOURCES:
        obj = os.path.join(build_dir, src + ".o")
        jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-pthread", "-ffp-contract=off", *inc, "-c",
                     os.path.join(CSRC, src), "-o", obj])
    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        outs = list(ex.map(_run, jobs))
    if verbose:
        for o in outs:
            sys.stdout.write(o)
    objs = [os.path.join(build_dir, s + ".o") for s in CUDA_SOURCES + CXX_SOURCES]
    tmp = lib_path + ".tmp"
    _run([nvcc, ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs, "-lpthread", "-ldl",
          "-Xlinker", "-rpath=" + os.path.join(cuda, "lib64")])
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, debug_bounds="--debug-bounds" in sys.argv))
