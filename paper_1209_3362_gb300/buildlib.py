"""Build the CUDA library libnfs_gb300.so in-tree with nvcc for sm_103a.

Every translation unit under csrc/ is compiled in parallel to an object file, then linked into a
shared library with the CUDA runtime linked statically.  Outputs go to
paper_1209_3362_gb300/_build/ (git-ignored).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libnfs_gb300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
              "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(ROOT, "include", "*.h")))


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


# Host-code sanitizers for a checking build (the host logic: schedules, band plans, bin tables,
# argument checks); device code is compiled as usual.
SANITIZE_FLAGS = ["-Xcompiler", "-fsanitize=address,-fsanitize=undefined,-fno-omit-frame-pointer", "-g"]


# Cycle accounting of the fused delay kernel's warp roles (nfs_delay_profile): a measuring build.
PROFILE_FLAGS = ["-DNFS_DELAY_PROFILE"]


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, sanitize: bool = False,
          profile: bool = False) -> str:
    """Compile every translation unit and link the library; returns its path.  sanitize=True builds
    a separate copy with AddressSanitizer and UBSan in the host code (loaded with libasan preloaded);
    profile=True a separate copy whose delay kernel accounts its warps' clock cycles by phase."""
    out = OUT + ("_sanitize" if sanitize else "") + ("_profile" if profile else "")
    lib = os.path.join(out, os.path.basename(LIB))
    os.makedirs(out, exist_ok=True)
    cc = nvcc()
    hdrs = _headers()
    jobs = []
    objs = []
    extra = (SANITIZE_FLAGS if sanitize else []) + (PROFILE_FLAGS if profile else [])
    for src in _sources():
        obj = os.path.join(out, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + hdrs):
            cmd = [cc, *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj]
            if ptxas_info:
                cmd += ["-Xptxas", "-v"]
            jobs.append(cmd)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        for cmd, r in ex.map(run, jobs):
            if verbose or ptxas_info or r.returncode:
                sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
            if r.returncode:
                raise RuntimeError(f"nvcc failed for {cmd[-3]}")
    if force or jobs or _stale(lib, objs):
        tmp = lib + f".{os.getpid()}.tmp"
        cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static", *(SANITIZE_FLAGS[:2] if sanitize else [])]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode:
            raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
