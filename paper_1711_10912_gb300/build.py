"""Builds libtlgb.so (the C-ABI CUDA library) in-tree for sm_103a.

Every .cu / .cpp file under csrc/ is compiled in parallel (nvcc for CUDA,
g++ for host C++) into _build/, then linked with nvcc into
paper_1711_10912_gb300/libtlgb.so.  A stamp holding the hash of the sources
and flags skips the build when nothing changed.  No cmake, no torch extension
machinery: the library is a plain shared object loaded through ctypes.
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libtlgb.so")
# the bounds-checked debug build (TL_CHECK_BOUNDS): every offset the index
# mappers produce is checked against its operand's extent; never the product
CHECKED_BUILD = os.path.join(ROOT, "_build_checked")
CHECKED_LIB = os.path.join(HERE, "libtlgb_checked.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
              "--expt-relaxed-constexpr", "-Xptxas", "-v"] + ARCH
CXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-Wall", "-Wextra", "-Wno-unused-parameter"]


def _nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return p


def _cuda_include() -> str:
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(_nvcc()))), "include")


def sources():
    out = []
    for f in sorted(os.listdir(CSRC)):
        if f.endswith((".cu", ".cpp")):
            out.append(os.path.join(CSRC, f))
    return out


def _digest(srcs, extra=()) -> str:
    h = hashlib.sha256()
    h.update(" ".join(extra).encode())
    for f in sorted(os.listdir(CSRC)) + [os.path.join("..", "..", "include", "tlgb.h")]:
        path = os.path.join(CSRC, f)
        if os.path.isfile(path):
            h.update(f.encode())
            with open(path, "rb") as fh:
                h.update(fh.read())
    h.update(" ".join(NVCC_FLAGS + CXX_FLAGS).encode())
    h.update(os.uname().machine.encode())
    return h.hexdigest()


def _compile(src: str, verbose: bool, build_dir: str = BUILD, extra=()):
    obj = os.path.join(build_dir, os.path.basename(src) + ".o")
    if src.endswith(".cu"):
        cmd = [_nvcc(), "-c", src, "-o", obj, "-I", CSRC, "-I", INCLUDE] + NVCC_FLAGS + list(extra)
    else:
        cmd = (["g++", "-c", src, "-o", obj, "-I", CSRC, "-I", INCLUDE, "-I", _cuda_include()] +
               CXX_FLAGS + list(extra))
    res = subprocess.run(cmd, capture_output=True, text=True)
    log = res.stdout + res.stderr
    if res.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{log}")
    if verbose and log.strip():
        sys.stderr.write(f"--- {os.path.basename(src)}\n{log}")
    return obj, log


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compiles and links libtlgb.so (or, with checked=True, the
    bounds-checked libtlgb_checked.so) if the sources changed; returns its
    path."""
    build_dir = CHECKED_BUILD if checked else BUILD
    lib = CHECKED_LIB if checked else LIB
    stamp = os.path.join(build_dir, os.path.basename(lib) + ".stamp")
    extra = ["-DTL_CHECK_BOUNDS"] if checked else []
    os.makedirs(build_dir, exist_ok=True)
    srcs = sources()
    dig = _digest(srcs, extra)
    if not force and os.path.exists(lib) and os.path.exists(stamp):
        with open(stamp) as fh:
            if fh.read().strip() == dig:
                return lib
    with ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose, build_dir, extra), srcs))
    objs = [o for o, _ in results]
    with open(os.path.join(build_dir, "ptxas.log"), "w") as fh:
        for o, log in results:
            fh.write(f"--- {os.path.basename(o)}\n{log}\n")
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [_nvcc(), "-shared", "-o", tmp] + objs + ARCH + ["-Xcompiler", "-fPIC"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{res.stdout}{res.stderr}")
    os.replace(tmp, lib)
    with open(stamp, "w") as fh:
        fh.write(dig)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                checked="--checked" in sys.argv))
