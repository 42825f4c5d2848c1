"""In-tree build of libvne.so (CUDA C++ for sm_103a) and the graph generator.

Each translation unit is compiled in parallel with nvcc
(``-gencode arch=compute_103a,code=sm_103a -lineinfo -O3``) and linked into
``paper_2212_09642_gb300/libvne.so`` with the CUDA runtime linked statically,
so the library does not depend on a runtime found at load time.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import platform
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libvne.so")
SOURCES = ["kernels_lanczos.cu", "kernels_dense.cu", "engine.cu", "abi.cu", "hutchpp.cu", "rational_driver.cu",
           "probing.cu", "batch.cu", "autotune.cu", "serve.cu", "host_graph.cpp", "noalloc.cu", "rational.cu",
           "assemble.cu", "measure.cu", "coloring.cu", "tcgen05_sketch.cu", "layout.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libvne")


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-pthread", "-I",
                   os.path.join(ROOT, "include"), "--expt-relaxed-constexpr"] + list(extra)


def _inputs_digest(extra) -> str:
    h = hashlib.sha256()
    for f in sorted(os.listdir(CSRC)):
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    with open(os.path.join(ROOT, "include", "vne.h"), "rb") as fh:
        h.update(fh.read())
    h.update(" ".join(_flags(extra)).encode())
    h.update(platform.machine().encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    """Compile libvne.so if its sources changed; return its path."""
    os.makedirs(BUILD, exist_ok=True)
    stamp = os.path.join(BUILD, "stamp")
    digest = _inputs_digest(extra)
    if not force and os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read() == digest:
        return LIB
    nvcc = nvcc_path()

    def compile_one(src):
        obj = os.path.join(BUILD, src + ".o")
        cmd = [nvcc, "-c", os.path.join(CSRC, src), "-o", obj] + _flags(extra)
        if src.endswith(".cpp"):
            cmd += ["-x", "cu"] if False else []
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "static", "-Xcompiler", "-pthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link of libvne.so failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as fh:
        fh.write(digest)
    return LIB


def build_all(verbose: bool = False) -> None:
    from . import graphs

    graphs.build_generator_library()
    build(verbose=verbose)


if __name__ == "__main__":
    build_all(verbose=True)
    print(LIB)
