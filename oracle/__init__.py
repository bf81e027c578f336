"""Plain FP64 CPU oracle for the structure function of dynamic NFS image sequences.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py``.  The CUDA library never imports, links or calls it, and the two share no
code.  The arithmetic lives in ``nfs_oracle.c`` (its header states the definition it follows:
the differential analysis and Eq. 1 of the paper, with the readings where the paper is silent);
this file only compiles it with gcc and marshals arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nfs_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libnfs_oracle.so")
_lib = None


def build(force: bool = False, sanitize: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP) into oracle/_build/libnfs_oracle.so; sanitize=True builds
    a separate copy with AddressSanitizer and UBSan (loaded with libasan preloaded)."""
    out = _LIB.replace(".so", "_sanitize.so") if sanitize else _LIB
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".{os.getpid()}.tmp"
        extra = ["-g", "-fsanitize=address,undefined", "-fno-omit-frame-pointer"] if sanitize else []
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-fopenmp", *extra,
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


def lib():
    """The compiled oracle (NFS_ORACLE_LIB names another build of the same source, e.g. a
    sanitizer build)."""
    global _lib
    if _lib is None:
        path = os.environ.get("NFS_ORACLE_LIB") or build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i = ctypes.c_int
        L.nfsor_fft2.argtypes = [i, i, P, P, P, P]
        L.nfsor_bins.argtypes = [i, i, i, P, P, P]
        L.nfsor_structure_function_u16.argtypes = [P, i, i, i, P, i, i, i, P, P, P, P, P]
        L.nfsor_structure_function_f64.argtypes = [P, i, i, i, i, P, i, i, i, P, P, P, P, P]
        L.nfsor_mode_power_u16.argtypes = [P, i, i, i, i, i, i, i, P]
        L.nfsor_max_threads.argtypes = []
        for f in (L.nfsor_fft2, L.nfsor_bins, L.nfsor_structure_function_u16, L.nfsor_structure_function_f64,
                  L.nfsor_mode_power_u16, L.nfsor_max_threads):
            f.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


def max_threads() -> int:
    return int(lib().nfsor_max_threads())


def fft2(a: np.ndarray) -> np.ndarray:
    """Unscaled forward 2-D DFT (sign e^{-i}) of a real or complex H x W array, full plane."""
    a = np.asarray(a)
    H, W = a.shape
    re = np.ascontiguousarray(a.real, dtype=np.float64)
    im = np.ascontiguousarray(a.imag if np.iscomplexobj(a) else np.zeros_like(re), dtype=np.float64)
    ore = np.empty((H, W), np.float64)
    oim = np.empty((H, W), np.float64)
    _check(lib().nfsor_fft2(H, W, _ptr(re), _ptr(im), _ptr(ore), _ptr(oim)), "fft2")
    return ore + 1j * oim


def bins(H: int, W: int, nq: int):
    """(bin_of_mode[H][W/2+1] int32 with -1 = excluded, C_b int64[nq], q_mean float64[nq])."""
    b = np.empty((H, W // 2 + 1), np.int32)
    c = np.empty(nq, np.int64)
    q = np.empty(nq, np.float64)
    _check(lib().nfsor_bins(H, W, nq, _ptr(b), _ptr(c), _ptr(q)), "bins")
    return b, c, q


def structure_function(frames: np.ndarray, delays: Sequence[int], nq: int, *, normalize: bool = True,
                       nthreads: int = 0, want_2d: bool = False) -> dict:
    """Binned D(q, tau) of a frame sequence [N, H, W] (uint16 counts or FP64 images).

    Returns dict(D[nd][nq], bin_counts[nq], pair_counts[nd], q_mean[nq], and D2d[nd][H][W/2+1] when
    want_2d).  uint16 frames are always normalised by their mean; FP64 frames only if normalize.
    """
    frames = np.ascontiguousarray(frames)
    N, H, W = frames.shape
    d = np.ascontiguousarray(np.asarray(delays, dtype=np.int32))
    nd = d.size
    D = np.zeros((nd, nq), np.float64)
    bc = np.zeros(nq, np.int64)
    pc = np.zeros(nd, np.int64)
    qm = np.zeros(nq, np.float64)
    D2 = np.zeros((nd, H, W // 2 + 1), np.float64) if want_2d else None
    if frames.dtype == np.uint16:
        rc = lib().nfsor_structure_function_u16(_ptr(frames), N, H, W, _ptr(d), nd, nq, nthreads, _ptr(D), _ptr(bc),
                                                _ptr(pc), _ptr(qm), _ptr(D2))
    else:
        f = np.ascontiguousarray(frames, dtype=np.float64)
        rc = lib().nfsor_structure_function_f64(_ptr(f), N, H, W, 1 if normalize else 0, _ptr(d), nd, nq,
                                                nthreads, _ptr(D), _ptr(bc), _ptr(pc), _ptr(qm), _ptr(D2))
    _check(rc, "structure_function")
    out = dict(D=D, bin_counts=bc, pair_counts=pc, q_mean=qm)
    if want_2d:
        out["D2d"] = D2
    return out


def mode_power(frames: np.ndarray, kx: int, ky: int, tau: int, nthreads: int = 0) -> float:
    """D(k, tau) at one half-plane mode of uint16 frames, by real-space differences."""
    frames = np.ascontiguousarray(frames, dtype=np.uint16)
    N, H, W = frames.shape
    out = np.zeros(1, np.float64)
    _check(lib().nfsor_mode_power_u16(_ptr(frames), N, H, W, kx, ky, tau, nthreads, _ptr(out)), "mode_power")
    return float(out[0])
