"""Host-side checks of the CUDA library that need no GPU: it loads, exports every symbol the public
header declares, and rejects bad arguments before touching the device."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import paper_1209_3362_gb300 as P


@pytest.fixture(scope="module")
def lib():
    P.build()
    return P.load_library()


def test_exports_every_header_symbol(lib):
    names = P.header_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    # and the dynamic symbol table agrees (extern "C", unmangled)
    out = subprocess.run(["nm", "-D", "--defined-only", P.LIB_PATH], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert set(names) <= exported


def test_binding_constants_match_the_header():
    """Every status, path, option, fit-method and stage constant of the binding equals the header's
    #define of the same name."""
    import re
    defs = {}
    for line in open(P.HEADER):
        m = re.match(r"#define (NFS_\w+) \(?(-?\d+)(?:ull)?\)?", line)
        if m:
            defs[m.group(1)] = int(m.group(2))
    pairs = {"NFS_OK": P.NFS_OK, "NFS_EINVAL": P.NFS_EINVAL, "NFS_EUNSUPPORTED": P.NFS_EUNSUPPORTED,
             "NFS_ENOMEM": P.NFS_ENOMEM, "NFS_ECUDA": P.NFS_ECUDA, "NFS_ESTATE": P.NFS_ESTATE,
             "NFS_ETOOBIG": P.NFS_ETOOBIG, "NFS_ETIMEOUT": P.NFS_ETIMEOUT,
             "NFS_PATH_FUSED_F32": P.PATH_FUSED_F32, "NFS_PATH_PLAIN_F64": P.PATH_PLAIN_F64,
             "NFS_FIT_GAUSS_NEWTON": P.FIT_GAUSS_NEWTON, "NFS_FIT_ADAM": P.FIT_ADAM,
             "NFS_N_STAGES": len(P.STAGES)}
    for name in ("TIMING", "BLOCK_FRAMES", "RING_SLOTS", "PITCH", "PATH", "FFT_CHUNK", "DELAY_VARIANT",
                 "FFT_GENERIC", "TEST_STALL_GROUP"):
        pairs["NFS_OPT_" + name] = getattr(P, "OPT_" + name)
    for i, st in enumerate(P.STAGES):
        assert defs["NFS_STAGE_" + st.upper()] == i, st
    for k, v in pairs.items():
        assert defs[k] == v, k
    assert (defs["NFS_NOALLOC_SCRATCH_BYTES"] << 20) == P.NOALLOC_SCRATCH_BYTES


def _create(lib, H, W, delays, nq, path=0, block=0):
    h = ctypes.c_void_p()
    d = np.ascontiguousarray(np.asarray(delays, np.int32))
    rc = lib.nfs_create_ex(H, W, d.ctypes.data if d.size else None, d.size, nq, path, block, ctypes.byref(h))
    return rc, h


@pytest.mark.parametrize("H,W", [(10, 64), (64, 10), (7, 8), (8, 7), (64, 8192), (0, 8), (5 * 64, 64),
                                 (64, 2 * 5)])
def test_rejects_unsupported_shapes(lib, H, W):
    rc, h = _create(lib, H, W, [1, 2], 8)
    assert rc in (P.NFS_EUNSUPPORTED, P.NFS_EINVAL) and not h.value


@pytest.mark.parametrize("delays,nq,path,block", [([2, 1], 8, 0, 0), ([1, 1], 8, 0, 0), ([-1, 2], 8, 0, 0),
                                                  ([], 8, 0, 0), ([1, 2], 0, 0, 0), ([1, 2], 8, 7, 0),
                                                  ([1, 2], 8, 0, 513), ([1, 70000], 8, 0, 0),
                                                  (list(range(1, 65537)), 8, 0, 0)])
def test_rejects_bad_arguments(lib, delays, nq, path, block):
    rc, h = _create(lib, 64, 64, delays, nq, path, block)
    assert rc == P.NFS_EINVAL and not h.value


def test_null_safety_and_status_text(lib):
    lib.nfs_destroy(None)
    assert lib.nfs_strerror(P.NFS_EUNSUPPORTED) == b"unsupported frame shape"
    assert lib.nfs_strerror(P.NFS_ECUDA) == b"CUDA error"
    assert lib.nfs_push_frames(None, None, 1) == P.NFS_EINVAL
    assert lib.nfs_structure_function(None, None, None, None, None) == P.NFS_EINVAL
    assert lib.nfs_frame_count(None) == -1
    assert lib.nfs_create(64, 64, None, 2, 8, ctypes.byref(ctypes.c_void_p())) == P.NFS_EINVAL


@pytest.mark.parametrize("H,W,nq", [(6, 8, 3), (48, 64, 24), (64, 96, 100), (2048, 2048, 1024),
                                    (4096, 3072, 1536), (486, 2048, 8000), (1458, 2048, 2100)])
def test_bin_table_equals_oracle(lib, oracle_lib, H, W, nq):
    """The library's radial bin table (host code of its own) equals the oracle's, bin for bin, also
    where 4 n_q^2 r2 passes 64 bits (the last two shapes)."""
    got = P.bin_table(H, W, nq)
    b, c, q = oracle_lib.bins(H, W, nq)
    np.testing.assert_array_equal(got["bin_of_mode"], b)
    np.testing.assert_array_equal(got["bin_counts"], c)
    np.testing.assert_allclose(got["q_mean"], q, rtol=1e-14, atol=0)


def test_noalloc_rejects_bins_beyond_64_bits(lib):
    """The no-allocation entry point's device bin index is 64-bit: n_q lcm(H, W) too large is
    refused before any GPU work (486 x 2048 frames, lcm 497,664, with 8000 bins)."""
    d = np.array([1, 2], np.int32)
    D = np.zeros((2, 8000)); bc = np.zeros(8000, np.int64); pc = np.zeros(2, np.int64)
    rc = lib.nfs_structure_function_noalloc(None, 0, 486, 2048, d.ctypes.data, 2, 8000, None, D.ctypes.data,
                                            bc.ctypes.data, pc.ctypes.data)
    assert rc == P.NFS_EUNSUPPORTED


def test_frame_count_limits(lib):
    """Frame indices in the kernels are 32-bit: the no-allocation entry point and the out-of-core
    driver refuse frame counts beyond their limits before touching memory or the GPU."""
    d = np.array([1, 2], np.int32)
    D = np.zeros((2, 8)); bc = np.zeros(8, np.int64); pc = np.zeros(2, np.int64)
    fake = ctypes.c_void_p(1 << 20)  # never dereferenced: the count is refused first
    assert lib.nfs_structure_function_noalloc(fake, (1 << 30) + 1, 64, 64, d.ctypes.data, 2, 8, None,
                                              D.ctypes.data, bc.ctypes.data, pc.ctypes.data) == P.NFS_EINVAL
    nt = ctypes.c_int64()
    assert lib.nfs_structure_function_out_of_core(64, 64, d.ctypes.data, 2, 8, fake, (1 << 31) - 1, 4096,
                                                  D.ctypes.data, bc.ctypes.data, pc.ctypes.data, None,
                                                  ctypes.byref(nt)) == P.NFS_EINVAL


def test_bin_table_rejects(lib):
    assert lib.nfs_bin_table(64, 64, 0, None, np.zeros(1, np.int64).ctypes.data, None) == P.NFS_EINVAL
    assert lib.nfs_bin_table(64, 64, 8, None, None, None) == P.NFS_EINVAL
    assert lib.nfs_bin_table(64, 70, 8, None, np.zeros(8, np.int64).ctypes.data, None) == P.NFS_EUNSUPPORTED


def _roi_create(lib, H, W, rois, delays=(1, 2, 5), nq=16):
    y0, x0, h, w = (np.ascontiguousarray(np.array([r[i] for r in rois], np.int32)) for i in range(4))
    d = np.ascontiguousarray(np.asarray(delays, np.int32))
    q = np.full(max(len(rois), 1), nq, np.int32)
    out = ctypes.c_void_p()
    rc = lib.nfs_roi_create(H, W, len(rois), y0.ctypes.data, x0.ctypes.data, h.ctypes.data, w.ctypes.data,
                            d.ctypes.data if d.size else None, d.size, q.ctypes.data, ctypes.byref(out))
    return rc, out


@pytest.mark.parametrize("H,W,rois,delays,nq,want", [
    (128, 128, [(0, 0, 64, 64), (100, 0, 64, 64)], (1, 2), 16, "EINVAL"),   # below the frame
    (128, 128, [(0, 70, 64, 64)], (1, 2), 16, "EINVAL"),                     # right of the frame
    (128, 128, [(-2, 0, 64, 64)], (1, 2), 16, "EINVAL"),
    (128, 128, [(0, 1, 64, 64)], (1, 2), 16, "EINVAL"),                      # odd x0
    (128, 128, [(0, 0, 64, 63)], (1, 2), 16, "EINVAL"),                      # odd w
    (128, 127, [(0, 0, 64, 64)], (1, 2), 16, "EINVAL"),                      # odd W
    (128, 128, [], (1, 2), 16, "EINVAL"),
    (128, 128, [(0, 0, 64, 64)], (2, 1), 16, "EINVAL"),                      # delays not increasing
    (128, 128, [(0, 0, 64, 64)], (), 16, "EINVAL"),
    (128, 128, [(0, 0, 64, 64)], (1, 2), 0, "EINVAL"),
    (128, 128, [(0, 0, 64, 64), (0, 0, 50, 64)], (1, 2), 16, "EUNSUPPORTED"),  # 50 = 2 x 5 x 5
    (128, 128, [(0, 0, 10, 64)], (1, 2), 16, "EUNSUPPORTED"),
])
def test_roi_create_rejects(lib, H, W, rois, delays, nq, want):
    rc, out = _roi_create(lib, H, W, rois, delays, nq)
    assert rc == getattr(P, "NFS_" + want) and not out.value


def test_roi_count_limit(lib):
    n = 65536
    z = np.zeros(n, np.int32)
    e = np.full(n, 8, np.int32)
    d = np.array([1, 2], np.int32)
    rc = lib.nfs_roi_create(64, 64, n, z.ctypes.data, z.ctypes.data, e.ctypes.data, e.ctypes.data, d.ctypes.data,
                            2, e.ctypes.data, ctypes.byref(ctypes.c_void_p()))
    assert rc == P.NFS_EINVAL


def test_roi_null_safety(lib):
    assert lib.nfs_roi_push(None, None, 0) == P.NFS_EINVAL
    assert lib.nfs_roi_push_device(None, None, 0) == P.NFS_EINVAL
    one = np.zeros(1, np.int32)
    assert lib.nfs_roi_create(64, 64, 1, None, one.ctypes.data, one.ctypes.data, one.ctypes.data, one.ctypes.data,
                              1, one.ctypes.data, ctypes.byref(ctypes.c_void_p())) == P.NFS_EINVAL
    assert lib.nfs_roi_create(64, 64, 1, one.ctypes.data, one.ctypes.data, one.ctypes.data, one.ctypes.data,
                              one.ctypes.data, 1, one.ctypes.data, None) == P.NFS_EINVAL


def test_no_cpu_fallback_in_product_path():
    """The package never imports the oracle: the product path has no CPU route."""
    import paper_1209_3362_gb300
    src_dir = os.path.dirname(paper_1209_3362_gb300.__file__)
    for root, _, files in os.walk(src_dir):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(root, f)).read()
                assert "import oracle" not in text and "from oracle" not in text and "nfsor_" not in text, f


# ---------------------------------------------------------------- out-of-core band plan (host logic)

def _block():
    return P.delay_schedule([1])["block_frames"]


def _check_plan(delays, N, Rmax):
    K = _block()
    p = P.out_of_core_plan(delays, N, Rmax)
    first, shift = list(p["band_first"]), list(p["band_shift"])
    assert first[0] == 0 and first[-1] == len(delays) and len(first) == len(shift) + 1
    assert all(a < b for a, b in zip(first, first[1:]))  # every delay in exactly one band, in order
    expect = 0
    for b, s in enumerate(shift):
        d = delays[first[b]:first[b + 1]]
        if s == 0:
            assert b == 0 and d[-1] + K <= Rmax  # in place: ring of d_max + K slots
            expect += N
        else:
            assert s % K == 0 and s == d[0] // K * K  # shifted pass: blocks stay on multiples of K
            assert (d[-1] - s) + 2 * K <= Rmax  # old-frame ring plus the K-slot current ring
            expect += 2 * max(0, N - s)
    assert p["n_transforms"] == expect
    return p


@pytest.mark.parametrize("Rmax", [3000, 2512, 2000, 1700, 1536])
def test_out_of_core_plan_log_delays(lib, Rmax):
    d = [int(x) for x in __import__("nfs_synth").log_delays(1, 2000, 200)]
    p = _check_plan(d, 4000, Rmax)
    if Rmax >= 2000 + _block():
        assert len(p["band_shift"]) == 1 and p["n_transforms"] == 4000  # fits: one ordinary pass


def test_out_of_core_plan_all_delays(lib):
    """All N - 1 delays (the paper's own case) with memory for N* spectra: the band passes make
    exactly N + sum 2 (N - s) transforms (checked in _check_plan).  The paper's FIFO scheme makes
    N (2 alpha - 3 + 2/alpha), alpha = (N - 1) / N*; the bands make more here (every shifted pass
    keeps two 512-frame blocks of slots and a band's schedule holds at most 4096 consecutive
    delays), the price of blocked, FMA-bound pair updates."""
    for N, Ns in ((16385, 8192), (8193, 2048), (4097, 2048)):
        p = _check_plan(list(range(1, N)), N, Ns)
        a = (N - 1) / Ns
        paper = N * (2 * a - 3 + 2 / a)
        assert paper <= p["n_transforms"] <= 6 * paper


def test_out_of_core_plan_random(lib):
    """Seeded delay lists and slot budgets: every plan the planner returns keeps the band invariants
    and the exact transform count (_check_plan), and every band's delays have a copy schedule for
    the fused kernel (ordinary for band 0, shifted for the others)."""
    K = _block()
    rng = np.random.Generator(np.random.PCG64(1209))
    planned = 0
    for _ in range(60):
        n = int(rng.integers(2, 300))
        d = np.cumsum(rng.integers(1, int(rng.choice([2, 8, 60, 400])), size=n))
        d = [int(x) for x in d if x <= 60000]
        N = int(d[-1] + rng.integers(1, 3000))
        Rmax = int(rng.integers(3 * K, 3 * K + 6000))
        try:
            p = _check_plan(d, N, Rmax)
        except P.NFSError:
            continue
        first, shift = list(p["band_first"]), list(p["band_shift"])
        for b, sft in enumerate(shift):
            sc = P.delay_schedule(d[first[b]:first[b + 1]], cross=sft > 0)
            assert len(sc["stages"]) >= 1
        planned += 1
    assert planned >= 40


def test_out_of_core_plan_rejects(lib):
    K = _block()
    with pytest.raises(P.NFSError):
        P.out_of_core_plan([1, 2, 6 * K - 2], 8 * K, 3 * K - 10)  # (d - s) + 2K > the budget: no band holds it
    with pytest.raises(P.NFSError):
        P.out_of_core_plan([5, 3], 100, 4000)  # not increasing
    p = P.out_of_core_plan([0, 1, 2], 10, K + 10)  # tau = 0 stays in the ordinary band
    assert list(p["band_first"]) == [0, 3] and p["n_transforms"] == 10
