"""Parity of the CUDA library with the FP64 oracle, element by element on the same seeded frames.

Tolerance: the fused FP32 path must match the oracle to 2e-5 relative on every binned D_b(tau)
whose bin and pair counts are non-zero; the plain FP64 path to 1e-12.  Bin and pair counts are
integers and must match exactly.  Empty entries must be exactly 0.
"""
import numpy as np
import pytest
import torch

import nfs_synth as S
import paper_1209_3362_gb300 as P

pytestmark = pytest.mark.gpu

TOL_F32 = 2e-5
TOL_F64 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    torch.cuda.init()
    P.build()
    P.load_library()


def rel_err(got, ref):
    D, R = got["D"], ref["D"]
    mask = (ref["bin_counts"][None, :] > 0) & (ref["pair_counts"][:, None] > 0)
    assert np.all(D[~mask] == 0.0)
    zero = mask & (R == 0.0)  # tau = 0 or identical frames: exact zero on both sides
    assert np.all(D[zero] == 0.0)
    mask &= R != 0.0
    if not mask.any():
        return 0.0
    return float(np.max(np.abs(D[mask] - R[mask]) / np.abs(R[mask])))


def check_counts(got, ref):
    np.testing.assert_array_equal(got["bin_counts"], ref["bin_counts"])
    np.testing.assert_array_equal(got["pair_counts"], ref["pair_counts"])
    np.testing.assert_allclose(got["q_mean"], ref["q_mean"], rtol=1e-12, atol=0)


def run_lib(frames, delays, nq, path="f32", block=0, chunks=None, device=False):
    with P.NFS(frames.shape[1], frames.shape[2], delays, nq, path=path, block_frames=block) as ctx:
        if device:
            ctx.push_frames_device(torch.from_numpy(frames.view(np.int16)).cuda())
        elif chunks is None:
            ctx.push_frames(frames)
        else:
            o = 0
            for c in chunks:
                ctx.push_frames(frames[o:o + c])
                o += c
            assert o == frames.shape[0]
        return ctx.structure_function()


@pytest.fixture(scope="module")
def ddm128(oracle_lib):
    w = S.WORKLOADS["ddm128"]
    fr = S.workload_source(w).frames_numpy(w.N)
    ref = oracle_lib.structure_function(fr, w.delays, w.n_qbins)
    return w, fr, ref


def test_ddm128_full_fused_f32(ddm128):
    w, fr, ref = ddm128
    got = run_lib(fr, w.delays, w.n_qbins)
    check_counts(got, ref)
    assert rel_err(got, ref) <= TOL_F32


def test_ddm128_full_plain_f64(ddm128):
    w, fr, ref = ddm128
    got = run_lib(fr, w.delays, w.n_qbins, path="f64")
    check_counts(got, ref)
    assert rel_err(got, ref) <= TOL_F64


@pytest.mark.parametrize("block", [1, 5, 17, 32])
def test_block_sizes(ddm128, block):
    w, fr, ref = ddm128
    got = run_lib(fr, w.delays, w.n_qbins, block=block)
    assert rel_err(got, ref) <= TOL_F32


def test_chunked_and_device_pushes_are_bit_identical(ddm128):
    w, fr, ref = ddm128
    a = run_lib(fr, w.delays, w.n_qbins)
    b = run_lib(fr, w.delays, w.n_qbins, chunks=[1, 7, 33, 2, 64, 50, 43])
    c = run_lib(fr, w.delays, w.n_qbins, device=True)
    np.testing.assert_array_equal(a["D"], b["D"])
    np.testing.assert_array_equal(a["D"], c["D"])


def test_running_result_and_reset(oracle_lib):
    fr = S.OUFrameSource(64, 96, 1.0, seed=21).frames_numpy(90)
    delays = [1, 2, 3, 7, 20, 41, 60]
    with P.NFS(64, 96, delays, 24) as ctx:
        ctx.push_frames(fr[:37])
        r1 = ctx.structure_function()
        assert rel_err(r1, oracle_lib.structure_function(fr[:37], delays, 24)) <= TOL_F32
        ctx.push_frames(fr[37:])
        r2 = ctx.structure_function()
        assert rel_err(r2, oracle_lib.structure_function(fr, delays, 24)) <= TOL_F32
        ctx.reset()
        ctx.push_frames(fr[10:70])
        r3 = ctx.structure_function()
        assert rel_err(r3, oracle_lib.structure_function(fr[10:70], delays, 24)) <= TOL_F32
        assert ctx.frame_count == 60


@pytest.mark.parametrize("path", ["f32", "f64"])
def test_empty_and_single_frame(oracle_lib, path):
    """No frames, an empty push and a single frame: every D is exactly 0 with pair count N - tau
    clipped at 0 (tau = 0 has one pair of identical frames); then two more frames match the oracle."""
    H, W, nq = 64, 64, 16
    delays = [0, 1, 2]
    fr = S.OUFrameSource(H, W, 1.0, seed=5).frames_numpy(3)
    _, counts, _ = oracle_lib.bins(H, W, nq)
    with P.NFS(H, W, delays, nq, path=path) as ctx:
        ctx.set_option(P.OPT_MODES, 1)  # every mode: the 2-D export below
        r0 = ctx.structure_function()
        assert np.all(r0["D"] == 0.0) and list(r0["pair_counts"]) == [0, 0, 0]
        np.testing.assert_array_equal(r0["bin_counts"], counts)
        ctx.push_frames(np.empty((0, H, W), np.uint16))
        ctx.push_frames_device(torch.empty((0, H, W), dtype=torch.int16, device="cuda"))
        ctx.push_frames(fr[:1])
        r1 = ctx.structure_function()
        assert np.all(r1["D"] == 0.0) and list(r1["pair_counts"]) == [1, 0, 0]
        assert np.all(ctx.export_spectrum(1) == 0.0)
        ctx.push_frames(fr[1:])
        r3 = ctx.structure_function()
    ref = oracle_lib.structure_function(fr, delays, nq)
    assert list(r3["pair_counts"]) == [3, 2, 1]
    assert np.all(r3["D"][0] == 0.0)
    assert rel_err(r3, ref) <= (TOL_F32 if path == "f32" else TOL_F64)


@pytest.mark.parametrize("H,W,nq,N,delays", [
    (8, 8, 4, 12, [0, 1, 2, 5, 11, 30]),
    (6, 8, 3, 9, [1, 2, 8]),
    (12, 16, 8, 20, [0, 1, 3, 19]),
    (6, 6, 3, 7, [1, 2]),
    (2, 2, 1, 5, [1, 2]),
    (16, 12, 40, 10, [1, 4]),
    (48, 64, 24, 40, [1, 2, 3, 4, 5, 10, 39]),
])
def test_edge_shapes(oracle_lib, H, W, nq, N, delays):
    fr = S.uniform_frames(N, H, W, seed=H * 1000 + W)
    ref = oracle_lib.structure_function(fr, delays, nq)
    for path, tol in (("f32", TOL_F32), ("f64", TOL_F64)):
        got = run_lib(fr, delays, nq, path=path)
        check_counts(got, ref)
        assert rel_err(got, ref) <= tol, path
        if delays[0] == 0:
            assert np.all(got["D"][0] == 0.0)


def test_identical_frames_give_exact_zero():
    fr = np.repeat(S.uniform_frames(1, 32, 32, seed=5), 40, axis=0)
    got = run_lib(fr, [1, 2, 17, 39, 45], 16)
    assert np.all(got["D"] == 0.0)
    assert list(got["pair_counts"]) == [39, 38, 23, 1, 0]


@pytest.mark.parametrize("H,W", [(384, 512), (96, 768), (768, 1024), (54, 2048), (6, 2048)])
def test_radix3_shapes(oracle_lib, H, W):
    """Radix-3 transform lengths, and 2048-wide frames whose heights are not a multiple of the row
    kernel's 4 rows per block (the one-warp-per-row 2048-wide row pass)."""
    fr = S.OUFrameSource(H, W, 2.0, seed=H + W).frames_numpy(10)
    delays = [1, 2, 5, 9]
    nq = min(H, W) // 2
    ref = oracle_lib.structure_function(fr, delays, nq)
    got = run_lib(fr, delays, nq)
    check_counts(got, ref)
    assert rel_err(got, ref) <= TOL_F32


def test_export_spectrum_matches_oracle_2d(oracle_lib):
    fr = S.OUFrameSource(32, 48, 1.0, seed=31).frames_numpy(40)
    delays = [1, 4, 13]
    ref = oracle_lib.structure_function(fr, delays, 16, want_2d=True)
    with P.NFS(32, 48, delays, 16) as ctx:
        ctx.set_option(P.OPT_MODES, 1)
        ctx.push_frames(fr)
        for j in range(len(delays)):
            got = ctx.export_spectrum(j)
            R = ref["D2d"][j]
            scale = np.mean(R)
            err = np.abs(got - R) / (np.abs(R) + 1e-3 * scale)
            assert err.max() <= 1e-4, (j, err.max())


def test_ddm1024_subset(oracle_lib):
    """Full 1024x1024 frames (the single-sequence workload's shape) on a short sequence."""
    w = S.WORKLOADS["ddm1024"]
    N = 24
    fr = S.OUFrameSource(w.H, w.W, w.Dc, seed=w.seed, device="cuda", dtype=torch.float32).frames_numpy(N)
    delays = [d for d in w.delays if d < N][:: 3] + [N - 1]
    delays = sorted(set(delays))
    ref = oracle_lib.structure_function(fr, delays, w.n_qbins)
    got = run_lib(fr, delays, w.n_qbins)
    check_counts(got, ref)
    assert rel_err(got, ref) <= TOL_F32


def _with_variant(frames, delays, nq, variant):
    with P.NFS(frames.shape[1], frames.shape[2], delays, nq) as ctx:
        ctx.set_option(P.OPT_DELAY_VARIANT, variant)
        ctx.push_frames(frames)
        return ctx.structure_function()


@pytest.fixture(scope="module")
def long64(oracle_lib):
    """1400 frames of 64x64 with log delays to 300: a full 512-frame block after the first
    tau_max + 512 frames (the unmasked steady-state kernel) and a ring of 812 slots that wraps."""
    fr = S.OUFrameSource(64, 64, 1.0, gamma0=0.01, seed=51).frames_numpy(1400)
    delays = S.log_delays(1, 300, 60)
    return fr, delays, oracle_lib.structure_function(fr, delays, 32)


def test_tiled_steady_state_and_ring_wrap(long64):
    fr, delays, ref = long64
    with P.NFS(64, 64, delays, 32) as ctx:
        K = ctx.get_option(P.OPT_BLOCK_FRAMES)
        assert K == 512 and 300 + 2 * K <= fr.shape[0]  # at least one block with every pair valid
        assert ctx.get_option(P.OPT_RING_SLOTS) == 300 + K < fr.shape[0]
        ctx.push_frames(fr)
        got = ctx.structure_function()
    check_counts(got, ref)
    assert rel_err(got, ref) <= TOL_F32


def test_delay_kernel_variants_agree(long64):
    fr, delays, ref = long64
    a = _with_variant(fr, delays, 32, 0)
    b = _with_variant(fr, delays, 32, 1)
    c = _with_variant(fr, delays, 32, 2)
    for x in (a, b, c):
        assert rel_err(x, ref) <= TOL_F32
    np.testing.assert_allclose(a["D"], b["D"], rtol=2e-6, atol=0)
    np.testing.assert_allclose(a["D"], c["D"], rtol=2e-6, atol=0)


def test_sparse_delays_with_large_gaps(oracle_lib):
    """Gaps wider than the shared-memory slot ring allows to prefetch across."""
    fr = S.OUFrameSource(32, 32, 3.0, seed=52).frames_numpy(1300)
    delays = [1, 2, 3, 400, 401, 900, 1250]
    ref = oracle_lib.structure_function(fr, delays, 16)
    got = run_lib(fr, delays, 16)
    check_counts(got, ref)
    assert rel_err(got, ref) <= TOL_F32


def test_specialised_and_generic_fft_agree_at_2048(oracle_lib):
    """2048x2048 frames (the paper-scale shape): size-specialised FFT kernels vs the generic ones,
    both against the oracle on a short sequence."""
    N = 6
    fr = S.OUFrameSource(2048, 2048, 1.0, gamma0=0.01, seed=61, device="cuda",
                         dtype=torch.float32).frames_numpy(N)
    delays = [1, 2, 5]
    ref = oracle_lib.structure_function(fr, delays, 1024)
    out = []
    for generic in (0, 1):
        with P.NFS(2048, 2048, delays, 1024) as ctx:
            ctx.set_option(P.OPT_FFT_GENERIC, generic)
            ctx.push_frames(fr)
            out.append(ctx.structure_function())
        check_counts(out[-1], ref)
        assert rel_err(out[-1], ref) <= TOL_F32, generic
    np.testing.assert_allclose(out[0]["D"], out[1]["D"], rtol=2e-6, atol=0)


def test_full_size_2048_sampled_modes(oracle_lib):
    """2048x2048 frames in the launch configuration the benchmark times (512-frame blocks, 32-frame
    FFT launches, steady-state blocks after tau_max): sampled modes of the exported 2-D spectra
    against the oracle's one-mode definition (real-space differences, one DFT coefficient), and
    the binned D against an FP64 re-binning of the exported spectra with the oracle's bin table."""
    H = W = 2048
    nq = 1024
    N = 840
    delays = [1, 2, 3, 4, 17, 180, 300]
    fr = S.OUFrameSource(H, W, 1.0, gamma0=0.01, seed=81, device="cuda", dtype=torch.float32).frames_numpy(N)
    with P.NFS(H, W, delays, nq) as ctx:
        K = ctx.get_option(P.OPT_BLOCK_FRAMES)
        assert K == 512 and ctx.get_option(P.OPT_FFT_CHUNK) == 32 and N >= delays[-1] + K  # a steady block
        ctx.set_option(P.OPT_MODES, 1)
        ctx.push_frames_device(torch.from_numpy(fr.view(np.int16)).cuda())
        got = ctx.structure_function()
        spectra = {j: ctx.export_spectrum(j) for j in (0, 1, 4, 6)}
    # the oracle, one mode at a time: low and high q, the k_x = 0 and k_x = W/2 columns, k_y > H/2
    samples = [(0, 3, 1), (5, 0, 4), (700, 1900, 6), (1024, 17, 0), (31, 1040, 4), (2, 2, 6)]
    for kx, ky, j in samples:
        ref = oracle_lib.mode_power(fr, kx, ky, delays[j])
        v = spectra[j][ky, kx]
        scale = float(np.mean(spectra[j]))
        assert abs(v - ref) / (abs(ref) + 1e-3 * scale) <= 1e-4, (kx, ky, delays[j], v, ref)
    # binning of the exported spectra (FP64, the oracle's integer bin rule and weights)
    b_of, counts, _ = oracle_lib.bins(H, W, nq)
    np.testing.assert_array_equal(got["bin_counts"], counts)
    w = np.full((H, W // 2 + 1), 2.0)
    w[:, 0] = 1.0
    w[:, W // 2] = 1.0
    keep = b_of >= 0
    for j, D2 in spectra.items():
        sums = np.bincount(b_of[keep], weights=(w * D2)[keep], minlength=nq)
        Db = np.where(counts > 0, sums / np.maximum(counts, 1), 0.0)
        np.testing.assert_allclose(got["D"][j], Db, rtol=1e-12, atol=0)
    assert np.all(got["pair_counts"] == [N - d for d in delays])
    assert np.all(got["D"] >= 0.0)


@pytest.mark.parametrize("path", ["f32", "f64"])
def test_dark_frames(oracle_lib, path):
    """Dark frames (every count 0) normalise to the zero image: dark frames at the start (the
    reference image then comes from the first lit frame) and in the middle of the sequence."""
    H, W, N, nq = 96, 128, 300, 48
    fr = S.OUFrameSource(H, W, 0.7, seed=77).frames_numpy(N).copy()
    fr[[0, 1, 2, 50, 51, 199]] = 0
    delays = [1, 2, 3, 48, 49, 150, 197]
    ref = oracle_lib.structure_function(fr, delays, nq)
    with P.NFS(H, W, delays, nq, path=path) as ctx:
        ctx.push_frames(fr)
        got = ctx.structure_function()
    np.testing.assert_array_equal(got["bin_counts"], ref["bin_counts"])
    np.testing.assert_array_equal(got["pair_counts"], ref["pair_counts"])
    assert np.all(np.isfinite(got["D"]))
    assert rel_err(got, ref) <= (TOL_F32 if path == "f32" else TOL_F64)


@pytest.mark.parametrize("H,W,path", [(4096, 4096, "f32"), (4096, 3072, "f32"), (4096, 4096, "f64")])
def test_max_frame_size(oracle_lib, H, W, path):
    """The largest frames the library takes (4096 rows; 4096 = the specialised 2048-point row
    transform, 3072 = the generic radix-3 row transform; 4096-point generic columns): sampled modes
    of the exported spectra against the oracle's one-mode definition, a delay with one pair only,
    and the binned D against an FP64 re-binning of the exported spectra."""
    nq = min(H, W) // 2
    N = 24
    delays = [1, 2, 7, 23]
    fr = S.OUFrameSource(H, W, 1.5, seed=4096 + W, device="cuda", dtype=torch.float32).frames_numpy(N)
    with P.NFS(H, W, delays, nq, path=path, block_frames=64 if path == "f32" else 0) as ctx:
        ctx.set_option(P.OPT_MODES, 1)
        ctx.push_frames(fr)
        got = ctx.structure_function()
        spectra = {j: ctx.export_spectrum(j) for j in range(len(delays))}
    tol = 1e-4 if path == "f32" else 1e-9
    samples = [(0, 3, 0), (5, 0, 1), (W // 2, 17, 2), (W // 2 - 648, 3000, 0), (31, H // 2 + 2, 3),
               (W // 2 - 1, H - 1, 1), (2, 2, 3)]
    for kx, ky, j in samples:
        ref = oracle_lib.mode_power(fr, kx, ky, delays[j])
        v = spectra[j][ky, kx]
        scale = float(np.mean(spectra[j]))
        assert abs(v - ref) / (abs(ref) + 1e-3 * scale) <= tol, (kx, ky, delays[j], v, ref)
    b_of, counts, _ = oracle_lib.bins(H, W, nq)
    np.testing.assert_array_equal(got["bin_counts"], counts)
    w = np.full((H, W // 2 + 1), 2.0)
    w[:, 0] = 1.0
    w[:, W // 2] = 1.0
    keep = b_of >= 0
    for j, D2 in spectra.items():
        sums = np.bincount(b_of[keep], weights=(w * D2)[keep], minlength=nq)
        Db = np.where(counts > 0, sums / np.maximum(counts, 1), 0.0)
        np.testing.assert_allclose(got["D"][j], Db, rtol=1e-12, atol=0)
    assert np.all(got["pair_counts"] == [N - d for d in delays])
    assert np.all(got["D"][:, counts > 0] > 0.0)


@pytest.mark.parametrize("Rmax", [2200, 1700])
def test_out_of_core_bands_match_in_core(oracle_lib, Rmax):
    """Out-of-core bands (each a pass over host frames with at most Rmax spectra on the device:
    an ordinary band, then shifted cross passes) give the in-core result bit for bit (every pair is
    added in the same block and order) and match the oracle; the passes transform exactly the
    planned frames."""
    fr = S.OUFrameSource(64, 64, 1.0, gamma0=0.01, seed=54).frames_numpy(3000)
    delays = S.log_delays(1, 2000, 70)
    plan = P.out_of_core_plan(delays, fr.shape[0], Rmax)
    assert len(plan["band_shift"]) >= 2 and plan["band_shift"][0] == 0
    got = P.structure_function_out_of_core(fr, delays, 32, Rmax)
    assert got["n_transforms"] == plan["n_transforms"]
    ref_gpu = run_lib(fr, delays, 32)
    np.testing.assert_array_equal(got["D"], ref_gpu["D"])
    np.testing.assert_array_equal(got["pair_counts"], ref_gpu["pair_counts"])
    ref = oracle_lib.structure_function(fr, delays, 32)
    check_counts(got, ref)
    assert rel_err(got, ref) <= TOL_F32


def test_all_delays_mode(oracle_lib):
    """Every delay 1..N-1 (the paper's own analysis): 128 sub-runs of 16 consecutive delays in the
    tiled kernel's schedule, pairs down to a single one at the largest delay."""
    N = 300
    fr = S.OUFrameSource(64, 64, 1.0, seed=55).frames_numpy(N)
    delays = list(range(1, N))
    ref = oracle_lib.structure_function(fr, delays, 32)
    got = run_lib(fr, delays, 32)
    check_counts(got, ref)
    assert got["pair_counts"][-1] == 1
    assert rel_err(got, ref) <= TOL_F32


def test_device_pushes_of_temporary_tensors():
    """Frames generated on the GPU and pushed as temporaries: generation may still be running on
    PyTorch's stream when the push is queued, and each tensor is dropped right after the call while
    the library still reads it on its own stream (its memory at once wanted by the next batch's
    generation).  The binding orders the library's stream after PyTorch's and keeps each tensor's
    memory until the library's stream has read it, so the result equals one push of a persistent
    tensor bit for bit."""
    H, W, N = 128, 192, 300
    delays, nq = [1, 2, 3, 10, 40, 200], 48
    src = S.OUFrameSource(H, W, 1.3, seed=91, device="cuda")
    frames = src.next_frames(N).clone()
    with P.NFS(H, W, delays, nq) as ctx:
        ctx.push_frames_device(frames)
        ref = ctx.structure_function()
    src = S.OUFrameSource(H, W, 1.3, seed=91, device="cuda")
    with P.NFS(H, W, delays, nq) as ctx:
        for o in range(0, N, 25):
            ctx.push_frames_device(src.next_frames(25))  # still being written, and freed when the call returns
        got = ctx.structure_function()
    np.testing.assert_array_equal(got["D"], ref["D"])


def test_delay_span_autotune_and_explicit_spans_are_bit_identical():
    """The stage span regroups the delay kernel's copy stages only: the autotuned span and explicit
    spans give the default's result bit for bit; the autotuner runs only before the first frame."""
    H, W, N = 96, 128, 1300
    delays, nq = S.log_delays(1, 1100, 60), 32
    dev = S.OUFrameSource(H, W, 0.9, seed=93, device="cuda").next_frames(N)
    results = {}
    for span in (None, 0, 64, 176, 512):
        with P.NFS(H, W, delays, nq) as ctx:
            if span is not None:
                ctx.set_option(P.OPT_DELAY_SPAN, span)
                got_span = ctx.get_option(P.OPT_DELAY_SPAN)
                assert got_span == span if span else got_span in (112, 176, 240, 320, 400)
            else:
                assert ctx.get_option(P.OPT_DELAY_SPAN) == 240
            ctx.push_frames_device(dev)
            results[span] = ctx.structure_function()
            if span == 0:
                with pytest.raises(P.NFSError) as e:
                    ctx.set_option(P.OPT_DELAY_SPAN, 0)
                assert e.value.status == P.NFS_ESTATE
            with pytest.raises(P.NFSError):
                ctx.set_option(P.OPT_DELAY_SPAN, 15)
    for span, r in results.items():
        np.testing.assert_array_equal(r["D"], results[None]["D"], err_msg=str(span))


def test_binned_modes_only_by_default(oracle_lib):
    """By default the FP32 delay update keeps only the 16-mode tiles that hold a binned mode (the
    corner modes beyond the Nyquist circle are in no bin): the binned result is bit-identical to a
    context that keeps every mode, the 2-D export asks for every mode, and the choice is made before
    the first frame.  Also checked on a slab context."""
    H, W, nq = 96, 128, 24
    fr = S.OUFrameSource(H, W, 1.2, seed=77).frames_numpy(700)
    delays = [1, 2, 3, 9, 40, 333]
    out = {}
    for modes in (0, 1):
        with P.NFS(H, W, delays, nq) as ctx:
            assert ctx.get_option(P.OPT_MODES) == 0
            ctx.set_option(P.OPT_MODES, modes)
            M = ctx.get_option(P.OPT_SLAB_MODES)
            kept = ctx.get_option(P.OPT_DELAY_MODES)
            assert (kept == M) if modes else (kept % 16 == 0 and 0.75 * M < kept < 0.9 * M)
            ctx.push_frames(fr[:300])
            with pytest.raises(P.NFSError) as e:
                ctx.set_option(P.OPT_MODES, 1 - modes)
            assert e.value.status == P.NFS_ESTATE
            ctx.push_frames(fr[300:])
            out[modes] = ctx.structure_function()
            if modes == 0:
                with pytest.raises(P.NFSError) as e:
                    ctx.export_spectrum(0)
                assert e.value.status == P.NFS_ESTATE
                assert ctx.structure_function()["pair_counts"][0] == 699  # the context is still usable
    np.testing.assert_array_equal(out[0]["D"], out[1]["D"])
    ref = oracle_lib.structure_function(fr, delays, nq)
    check_counts(out[0], ref)
    assert rel_err(out[0], ref) <= TOL_F32
    with P.NFS(H, W, delays, nq, slab=1, n_slabs=3) as c:
        c.push_frames(fr)
        slab = c.structure_function()
    with P.NFS(H, W, delays, nq, slab=1, n_slabs=3) as c:
        c.set_option(P.OPT_MODES, 1)
        c.push_frames(fr)
        np.testing.assert_array_equal(c.structure_function()["D"], slab["D"])

