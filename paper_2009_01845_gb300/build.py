"""Build libqsim_gb300.so in-tree with nvcc for sm_103a.

Every translation unit under ``csrc/`` is compiled in parallel with
``-gencode arch=compute_103a,code=sm_103a`` and linked into one shared library
at ``paper_2009_01845_gb300/_build/libqsim_gb300.so`` (with NVRTC, which
compiles pass kernels specialised at run time from the device headers, whose
texts are embedded). Rebuilds only when a source or header is newer than the
library.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libqsim_gb300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libqsim_gb300.so")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _deps():
    return sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        [os.path.join(INCLUDE, "qsim.h"), os.path.abspath(__file__)]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _deps())


# headers the run-time pass specialisation (csrc/tile_jit.cpp) hands to NVRTC
JIT_HEADERS = [("qsim_h", os.path.join(INCLUDE, "qsim.h")), ("device_cuh", os.path.join(CSRC, "device.cuh")),
               ("tiled_h", os.path.join(CSRC, "tiled.h")), ("tile_device_cuh", os.path.join(CSRC, "tile_device.cuh"))]


def write_jit_headers() -> None:
    """_build/jit_headers.inc: each header's text as a NUL-terminated char array
    kJitSrc_<name> (byte values, so no string-literal length limit applies)."""
    out = []
    for name, path in JIT_HEADERS:
        with open(path, "rb") as f:
            data = f.read()
        body = ",".join(str(b) for b in data + b"\0")
        out.append(f"static const char kJitSrc_{name}[] = {{{body}}};\n")
    tmp = os.path.join(BUILD, f"jit_headers.inc.tmp{os.getpid()}")
    with open(tmp, "w") as f:
        f.write("".join(out))
    os.replace(tmp, os.path.join(BUILD, "jit_headers.inc"))


def cuda_lib_dir() -> str:
    root = os.path.dirname(os.path.dirname(os.path.realpath(nvcc())))
    for d in (os.path.join(root, "lib64"), os.path.join(root, "lib")):
        if os.path.exists(os.path.join(d, "libnvrtc.so")):
            return d
    return os.path.join(root, "lib64")


def _compile(src: str, extra) -> str:
    obj = os.path.join(BUILD, os.path.basename(src) + ".o")
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
           "-I", INCLUDE, "-I", CSRC, "-I", BUILD, "--expt-relaxed-constexpr", *extra, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
    return obj


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    write_jit_headers()
    srcs = sources()
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda s: _compile(s, list(extra)), srcs))
    tmp = LIB + f".tmp{os.getpid()}"
    libdir = cuda_lib_dir()
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-L", libdir, "-lnvrtc", "-Xlinker", f"-rpath={libdir}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        print(f"built {LIB}", file=sys.stderr)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
