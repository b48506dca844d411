"""Build the engine library (CUDA, sm_103a) in-tree: paper_2605_28400_gb300/_lib/libtrioseq.so.

The translation units (host runtime, kernels, the semi-global/local, packed int16x2 and slab
kernel instantiations, the allocation-free entry) are compiled in parallel with nvcc for
sm_103a only, then linked into one shared library with the static CUDA runtime. No torch
extension machinery is involved; the Python side loads the library with ctypes.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
import threading
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libtrioseq.so")
SOURCES = ["runtime.cu", "kernels.cu", "kernels_variants.cu", "kernels_packed.cu",
           "kernels_slab.cu", "noalloc.cu", "alu_rate.cu", "kernels_vl.cu", "partition.cu",
           "affine.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
_lock = threading.Lock()


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the engine")


def _inputs():
    files = [os.path.join(CSRC, s) for s in SOURCES]
    files += [os.path.join(CSRC, "engine.h"), os.path.join(CSRC, "wavefront.cuh"),
              os.path.join(CSRC, "guard.h"),
              os.path.join(CSRC, "wavefront_vl.cuh"),
              os.path.join(ROOT, "include", "trioseq.h")]
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile if any source is newer than the library; returns the library path."""
    with _lock:
        if not force and up_to_date():
            return LIB
        os.makedirs(LIBDIR, exist_ok=True)
        cc = nvcc()
        flags = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
                        "-I", os.path.join(ROOT, "include"), "-I", CSRC]
        if verbose:
            flags += ["-Xptxas", "-v"]
        objs = []
        tag = f"{os.getpid()}"

        def comp(src):
            obj = os.path.join(LIBDIR, src.replace(".cu", f".{tag}.o"))
            cmd = [cc] + flags + ["-c", os.path.join(CSRC, src), "-o", obj]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
            if verbose:
                sys.stderr.write(r.stderr)
            return obj

        every = [os.path.join(LIBDIR, src.replace(".cu", f".{tag}.o")) for src in SOURCES]
        tmp = LIB + f".{tag}.tmp"
        try:
            with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
                objs = list(ex.map(comp, SOURCES))
            cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
            os.replace(tmp, LIB)
        finally:  # no objects or partial library left behind, whether or not the build worked
            for f in every + [tmp]:
                try:
                    os.remove(f)
                except OSError:
                    pass
        return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
