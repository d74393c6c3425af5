"""In-tree build of the CUDA library libgeomhd.so for sm_103a (nvcc, no cmake).

The translation units compile in parallel, then link into
paper_1905_02504_gb300/lib/libgeomhd.so.  Rebuilds only when a source is newer
than the library.
"""
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
INC = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIBDIR = os.path.join(HERE, "lib")
LIB = os.path.join(LIBDIR, "libgeomhd.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["host_tables.cpp", "kernels.cu", "api.cu", "noalloc.cu"]


def _refpattern():
    """The generator of refpattern.h (loaded by path: this file also runs as a script)."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("_geomhd_refpattern", os.path.join(HERE, "refpattern.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _nvcc():
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    path = os.path.join(cuda, "bin", "nvcc")
    return path if os.path.exists(path) else "nvcc"


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-fopenmp,-O3",
                   "-I" + INC, "-I" + SRC, "-I" + BUILD] + list(extra)


def _deps():
    files = [os.path.join(SRC, f) for f in os.listdir(SRC)] + [os.path.join(HERE, "refpattern.py")]
    files += [os.path.join(INC, f) for f in os.listdir(INC)]
    return files


def needs_build():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in _deps())


def build(verbose=False, ptxas_info=False, force=False):
    if not force and not needs_build():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    _refpattern().write(os.path.join(BUILD, "refpattern.h"))
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD, src + ".o")
        extra = ["-Xptxas", "-v"] if (ptxas_info and src.endswith(".cu")) else []
        cmd = [nvcc] + _flags(extra) + ["-c", os.path.join(SRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        if verbose or ptxas_info:
            print(r.stdout, r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp"
    cmd = [nvcc] + ARCH + ["-shared", "-Xcompiler", "-fopenmp", "-o", tmp] + objs + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(verbose=True, ptxas_info="-v" in sys.argv, force="-f" in sys.argv))
