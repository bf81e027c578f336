"""The library's host logic and the oracle under AddressSanitizer and UBSan (no GPU): copies built
with sanitize=True run the copy-schedule export, the band planner, the bin table and the argument
checks of the creating calls, and the oracle's transforms, bins and structure functions, on seeded
inputs in child processes with libasan preloaded; any out-of-bounds access, use after free or
undefined behaviour ends that process with an error."""
import os
import shutil
import subprocess
import sys

import pytest

import paper_1209_3362_gb300 as P
from paper_1209_3362_gb300 import buildlib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

DRIVER = r'''
import ctypes, sys
import numpy as np
sys.path.insert(0, ROOT)
import paper_1209_3362_gb300 as P
import nfs_synth as S
L = P.load_library(LIB)
P._lib = L
rng = np.random.Generator(np.random.PCG64(99))
for it in range(300):
    kind = it % 4
    if kind == 0:
        d = np.cumsum(rng.integers(1, 300, size=int(rng.integers(1, 300))))
    elif kind == 1:
        d = np.arange(1, int(rng.integers(2, 5000)))
    elif kind == 2:
        d = np.array(S.log_delays(1, int(rng.integers(10, 6000)), int(rng.integers(5, 300))))
    else:
        d = rng.integers(-3, 70000, size=int(rng.integers(0, 50)))
    d = np.ascontiguousarray(d.astype(np.int32))
    for cross in (False, True):
        try:
            P.delay_schedule(d, cross)
        except P.NFSError:
            pass
    try:
        P.out_of_core_plan(d, int(rng.integers(1, 20000)), int(rng.integers(1, 9000)))
    except P.NFSError:
        pass
for H, W, nq in [(6, 8, 3), (64, 96, 100), (486, 2048, 8000), (2048, 2048, 1024), (4096, 3072, 1536),
                 (2, 2, 1), (2, 4096, 65536)]:
    P.bin_table(H, W, nq)
for it in range(300):
    H = int(rng.choice([0, 2, 7, 64, 96, 4096, 5000])); W = int(rng.choice([0, 2, 9, 64, 96, 4096, 8192]))
    d = np.ascontiguousarray(rng.integers(-2, 100, size=int(rng.integers(0, 8))).astype(np.int32))
    h = ctypes.c_void_p()
    rc = L.nfs_create_ex(H, W, d.ctypes.data if d.size else None, d.size, int(rng.integers(-1, 70000)),
                         int(rng.integers(-1, 3)), int(rng.integers(-1, 600)), ctypes.byref(h))
    if rc == 0:
        L.nfs_destroy(h)
    rois = rng.integers(-4, 200, size=(int(rng.integers(0, 4)), 4)).astype(np.int32)
    cols = [np.ascontiguousarray(rois[:, i]) for i in range(4)]
    q = np.full(max(len(rois), 1), 8, np.int32)
    L.nfs_roi_create(H, W, len(rois), *[c.ctypes.data for c in cols], d.ctypes.data if d.size else None, d.size,
                     q.ctypes.data, ctypes.byref(h))
print("clean")
'''


def _libasan():
    gcc = shutil.which("gcc")
    if not gcc:
        return None
    p = subprocess.run([gcc, "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    return p if os.path.isabs(p) and os.path.exists(p) else None


def test_host_logic_under_sanitizers(tmp_path):
    asan = _libasan()
    if asan is None or shutil.which("nvcc") is None:
        pytest.skip("gcc's libasan or nvcc is not available")
    lib = buildlib.build(sanitize=True)
    script = tmp_path / "drive.py"
    script.write_text(f"ROOT = {ROOT!r}\nLIB = {lib!r}\n" + DRIVER)
    env = dict(os.environ, LD_PRELOAD=asan, ASAN_OPTIONS="detect_leaks=0",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1")
    r = subprocess.run([sys.executable, str(script)], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0 and "clean" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]


ORACLE_DRIVER = r'''
import sys
import numpy as np
sys.path.insert(0, ROOT)
import oracle
import nfs_synth as S
rng = np.random.Generator(np.random.PCG64(5))
for H, W in [(6, 8), (12, 16), (9, 6), (24, 32)]:
    a = rng.standard_normal((H, W)) + 1j * rng.standard_normal((H, W))
    assert np.allclose(oracle.fft2(a), np.fft.fft2(a))
for H, W, nq in [(6, 8, 3), (486, 2048, 8000), (64, 96, 100)]:
    oracle.bins(H, W, nq)
fr = S.uniform_frames(9, 12, 16, seed=3)
fr[4] = 0  # a dark frame
oracle.structure_function(fr, [0, 1, 2, 8, 20], 8, want_2d=True)
oracle.structure_function(fr.astype(np.float64), [1, 3], 6, normalize=False)
oracle.mode_power(fr, 3, 5, 2)
print("clean")
'''


def test_oracle_under_sanitizers(tmp_path):
    asan = _libasan()
    if asan is None:
        pytest.skip("gcc's libasan is not available")
    import oracle
    lib = oracle.build(sanitize=True)
    script = tmp_path / "drive_oracle.py"
    script.write_text(f"ROOT = {ROOT!r}\n" + ORACLE_DRIVER)
    env = dict(os.environ, LD_PRELOAD=asan, ASAN_OPTIONS="detect_leaks=0", NFS_ORACLE_LIB=lib,
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1", OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, str(script)], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0 and "clean" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]
