"""Build the CUDA library libfea.so in-tree with nvcc (sm_103a only).

Translation units are compiled in parallel and linked into one shared library
next to this file.  Rebuilds only when a source is newer than the library.
"""
import concurrent.futures
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libfea.so")
BUILD = os.path.join(HERE, "_build")
SOURCES = ["fea_api.cu", "batch.cu", "kernels_pre.cu", "kernels_se.cu", "kernels_naive.cu", "kernels_vec.cu", "kernels_tc.cu", "kernels_pretc.cu", "global.cu",
           "bernstein.cu",
           "host_model.cpp", "planner.cpp", "opcount.cpp", "theta.cpp", "mlp.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(os.path.dirname(HERE), "include", "fea.h"))
    return files


def needs_build():
    if not os.path.exists(OUT):
        return True
    t = os.path.getmtime(OUT)
    return any(os.path.getmtime(f) > t for f in _deps() + [os.path.abspath(__file__)])


def _compile(src):
    obj = os.path.join(BUILD, src + ".o")
    path = os.path.join(CSRC, src)
    cmd = [_nvcc(), *ARCH, "-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
           "-ftz=true", "-prec-div=true", "-prec-sqrt=true", "-fmad=true",
           "-I", CSRC, "-c", path, "-o", obj]
    if src.endswith(".cpp"):
        cmd = [_nvcc(), "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-I", CSRC, "-c", path, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
    return obj


def build(force=False, verbose=False):
    if not force and not needs_build():
        return OUT
    os.makedirs(BUILD, exist_ok=True)
    workers = min(len(SOURCES), max(2, os.cpu_count() or 2))
    with concurrent.futures.ThreadPoolExecutor(workers) as ex:
        objs = list(ex.map(_compile, SOURCES))
    tmp = OUT + ".%d.tmp" % os.getpid()
    cmd = [_nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s" % r.stderr)
    os.replace(tmp, OUT)
    if verbose:
        print("built", OUT, file=sys.stderr)
    return OUT


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
