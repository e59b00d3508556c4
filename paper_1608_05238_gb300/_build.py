"""In-tree build of libmcr.so (the sm_103a CUDA library behind include/mcr.h).

Compiles each translation unit under csrc/ with nvcc for sm_103a in parallel and links them
into ``paper_1608_05238_gb300/libmcr.so``.  No cmake, no torch extension machinery: the library
is a plain C-ABI shared object loaded with ctypes.

It also links ``libmcr_checked.so``: the transport library (the ``mcr*.cu`` units, not the
denoiser's) compiled with ``-DMCR_CHECKED``, in which every tally, medium and record index is
range-checked and every deposit checked for a finite weight on the device; a failed check skips
the access and latches MCR_ERR_CHECK (the tests run it where a memory checker is not available).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(os.path.dirname(PKG), "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libmcr.so")
LIB_CHECKED = os.path.join(PKG, "libmcr_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    cand = os.path.join(home, "bin", "nvcc")
    return cand if os.path.exists(cand) else (shutil.which("nvcc") or cand)


def sources() -> list[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _deps() -> list[str]:
    files = sources() + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    return files + [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]


def up_to_date() -> bool:
    if not (os.path.exists(LIB) and os.path.exists(LIB_CHECKED)):
        return False
    t = min(os.path.getmtime(LIB), os.path.getmtime(LIB_CHECKED))
    return all(os.path.getmtime(f) <= t for f in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile csrc/*.cu for sm_103a and link libmcr.so; returns its path."""
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE]
    if verbose:
        common += ["-Xptxas", "-v"]

    os.makedirs(os.path.join(BUILD, "checked"), exist_ok=True)

    def compile_one(job) -> str:
        src, checked = job
        obj = os.path.join(BUILD, "checked" if checked else "", os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc, *common, *(["-DMCR_CHECKED"] if checked else []), "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    srcs = sources()
    checked_srcs = [f for f in srcs if os.path.basename(f).startswith("mcr")]
    jobs = [(f, False) for f in srcs] + [(f, True) for f in checked_srcs]
    with cf.ThreadPoolExecutor(max_workers=max(1, min(16, os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_one, jobs))
    cuda_lib = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "lib64")
    for lib, lib_objs in ((LIB, objs[:len(srcs)]), (LIB_CHECKED, objs[len(srcs):])):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *lib_objs, "-Xlinker", f"-rpath,{cuda_lib}"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link of {os.path.basename(lib)} failed:\n{r.stderr}")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
