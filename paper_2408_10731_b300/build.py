"""Build libtrajbatch.so in-tree with nvcc for sm_103a (B300).

Each .cu file compiles to its own object in _lib/obj (in parallel; an object is
rebuilt when its source, a header or the flags are newer), then one link step
writes _lib/libtrajbatch.so. The translation units call each other only through
host launch wrappers, so no relocatable device code is needed.
"""
import glob
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "_lib", "libtrajbatch.so")
OBJ = os.path.join(HERE, "_lib", "obj")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC"]


def sources():
    return sorted(glob.glob(os.path.join(HERE, "csrc", "*.cu")))


def headers():
    return sorted(glob.glob(os.path.join(HERE, "csrc", "*.cuh"))) + \
        sorted(glob.glob(os.path.join(HERE, "csrc", "*.h"))) + \
        [os.path.join(ROOT, "include", "trajbatch.h"), os.path.abspath(__file__)]


def deps():
    return sources() + headers()


def _obj(src):
    return os.path.join(OBJ, os.path.basename(src)[:-3] + ".o")


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in deps())


def _compile(src, verbose):
    out = _obj(src)
    newest = max(os.path.getmtime(d) for d in [src] + headers())
    if os.path.exists(out) and os.path.getmtime(out) >= newest:
        return out
    cmd = [NVCC] + FLAGS + (["-Xptxas=-v"] if verbose else []) + \
        ["-I", os.path.join(ROOT, "include"), "-c", src, "-o", out + ".tmp"]
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    return out


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OBJ, exist_ok=True)
    if force:
        for s in sources():
            if os.path.exists(_obj(s)):
                os.remove(_obj(s))
    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose), sources()))
    tmp = LIB + ".tmp"
    subprocess.run([NVCC] + ARCH + ["-shared", "-o", tmp] + objs, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
