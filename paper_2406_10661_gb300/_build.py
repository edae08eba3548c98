"""Build steps for the compiled parts (nvcc for sm_103a, gcc for the C helper)."""
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
NVCC_FLAGS = ["-std=c++17", "-O3", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo",
              "-Xcompiler", "-fPIC", "-Xcompiler", "-pthread", "-shared"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _stale(out, srcs):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(s) > t for s in srcs)


def build_cuda(force=False, extra=()):
    out = os.path.join(HERE, "libmoss.so")
    units = ("moss_api.cu", "moss_noalloc.cu")
    srcs = [os.path.join(CSRC, f) for f in units + ("moss_device.cuh", "moss_kernels.cuh")]
    srcs.append(os.path.join(ROOT, "include", "moss.h"))
    if force or _stale(out, srcs):
        tmp = out + f".{os.getpid()}.tmp"
        subprocess.check_call([_nvcc(), *NVCC_FLAGS, *extra, "-I", os.path.join(ROOT, "include"),
                               "-o", tmp, *[os.path.join(CSRC, u) for u in units]])
        os.replace(tmp, out)
    return out


def build_route_walk(force=False):
    out = os.path.join(HERE, "_route_walk.so")
    src = os.path.join(CSRC, "route_walk.c")
    if force or _stale(out, [src]):
        tmp = out + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-pthread", "-o", tmp, src])
        os.replace(tmp, out)
    return out


def build_all(force=False):
    with ThreadPoolExecutor(2) as ex:
        a = ex.submit(build_cuda, force)
        b = ex.submit(build_route_walk, force)
        return a.result(), b.result()
