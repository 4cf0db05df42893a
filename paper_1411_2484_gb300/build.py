"""Build libphprng.so in-tree with nvcc for sm_103a (GB300).

Each translation unit under csrc/ is compiled in parallel, then linked into
paper_1411_2484_gb300/libphprng.so (CUDA runtime linked statically, only the
C ABI of include/phprng.h exported).  Rebuilds only when a source is newer
than the library.  ``python -m paper_1411_2484_gb300.build --ptxas-v`` also
prints register and shared-memory use per kernel.
"""
import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libphprng.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-fvisibility=hidden",
         "-I", os.path.join(ROOT, "include")]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _deps():
    return sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) \
        + [os.path.join(ROOT, "include", "phprng.h"), os.path.abspath(__file__)]


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _deps())


def _compile(src, ptxas_v, extra=(), obj_dir=OBJ):
    obj = os.path.join(obj_dir, os.path.basename(src) + ".o")
    cmd = [NVCC] + ARCH + FLAGS + list(extra) + (["-Xptxas", "-v"] if ptxas_v else []) + \
        ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
    return obj, r.stderr


def build(force=False, ptxas_v=False, verbose=False, defines=(), out=None):
    """Compile and link libphprng.so (or `out`, with extra -D `defines`)."""
    lib = out or LIB
    if not force and not ptxas_v and not defines and out is None and up_to_date():
        return LIB
    obj_dir = OBJ if out is None else out + ".objs"
    os.makedirs(obj_dir, exist_ok=True)
    srcs = sources()
    extra = ["-D" + d for d in defines]
    with ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        results = list(ex.map(lambda s: _compile(s, ptxas_v, extra, obj_dir), srcs))
    if ptxas_v or verbose:
        for (_, log), s in zip(results, srcs):
            if log.strip():
                print("==", os.path.basename(s))
                print(log)
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in results] + ["-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    build(force=True, ptxas_v="--ptxas-v" in sys.argv, verbose=True)
    print(LIB)
