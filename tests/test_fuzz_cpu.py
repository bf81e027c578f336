"""Seeded argument fuzzing of the C ABI's host-side entry points (no GPU): every call returns one
of the documented status codes, never crashes, and the host-only functions (schedule export, band
planner, bin table) either succeed or refuse their arguments consistently."""
import ctypes

import numpy as np
import pytest

import paper_1209_3362_gb300 as P

CODES = {P.NFS_OK, P.NFS_EINVAL, P.NFS_EUNSUPPORTED, P.NFS_ENOMEM, P.NFS_ECUDA, P.NFS_ESTATE, P.NFS_ETOOBIG}


@pytest.fixture(scope="module")
def lib():
    P.build()
    return P.load_library()


def _delays(rng):
    kind = int(rng.integers(0, 5))
    n = int(rng.integers(0, 40))
    if kind == 0:  # valid, increasing
        return np.cumsum(rng.integers(1, 300, size=n)).astype(np.int32)
    if kind == 1:  # arbitrary integers (negative, repeated, unsorted, huge)
        return rng.integers(-5, 70000, size=n).astype(np.int32)
    if kind == 2:  # starts at zero
        return np.concatenate([[0], np.cumsum(rng.integers(1, 50, size=n))]).astype(np.int32)
    if kind == 3:  # empty
        return np.zeros(0, np.int32)
    return np.array([int(rng.integers(1, 4000))] * max(n, 2), np.int32)  # repeated


def test_fuzz_host_entry_points(lib):
    rng = np.random.Generator(np.random.PCG64(13))
    for _ in range(400):
        d = np.ascontiguousarray(_delays(rng))
        dp = d.ctypes.data if d.size else None
        H = int(rng.choice([0, 2, 6, 7, 10, 48, 64, 96, 128, 4096, 5000, -4]))
        W = int(rng.choice([0, 2, 8, 9, 12, 64, 96, 4096, 8192, -2]))
        nq = int(rng.choice([-1, 0, 1, 3, 64, 65536, 70000]))
        # schedule export (host only)
        sr = np.zeros((64, 3), np.int32)
        st = np.zeros((64, 5), np.int32)
        outs = [ctypes.c_int(0) for _ in range(5)]
        span = int(rng.choice([0, 0, 15, 16, 100, 240, 512, 513, -1]))
        rc = lib.nfs_delay_schedule(dp, int(d.size), int(rng.integers(0, 2)), sr.ctypes.data, st.ctypes.data, 64,
                                    *[ctypes.byref(o) for o in outs], span)
        assert rc in CODES
        valid = (d.size > 0 and d[0] >= 0 and d[-1] <= 65536 and bool(np.all(np.diff(d) > 0))
                 and (span == 0 or 16 <= span <= 512))
        if not valid:
            assert rc == P.NFS_EINVAL
        # band planner (host only)
        first = np.zeros(d.size + 1, np.int32)
        shift = np.zeros(max(d.size, 1), np.int64)
        nb = ctypes.c_int(0)
        nt = ctypes.c_int64(0)
        rc = lib.nfs_out_of_core_plan(dp, int(d.size), int(rng.integers(-2, 6000)), int(rng.integers(-1, 9000)),
                                      first.ctypes.data, shift.ctypes.data, ctypes.byref(nb), ctypes.byref(nt))
        assert rc in CODES
        if rc == P.NFS_OK:
            assert 1 <= nb.value <= d.size and first[0] == 0 and first[nb.value] == d.size
        # bin table (host only; small shapes so the loop stays fast)
        if 0 < H <= 128 and 0 < W <= 128:
            c = np.zeros(max(nq, 1), np.int64)
            rc = lib.nfs_bin_table(H, W, nq, None, c.ctypes.data, None)
            assert rc in CODES
            if rc == P.NFS_OK:
                assert c.sum() > 0 or nq >= 1
        # context creation: argument errors come before any CUDA call
        h = ctypes.c_void_p()
        rc = lib.nfs_create_ex(H, W, dp, int(d.size), nq, int(rng.integers(-1, 3)), int(rng.integers(-1, 600)),
                               ctypes.byref(h))
        assert rc in CODES
        if rc == P.NFS_OK:
            lib.nfs_destroy(h)
        else:
            assert not h.value
