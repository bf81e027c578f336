"""Pins of the FP64 oracle against what mathematics and the paper fix (CPU only).

Each test would fail under a plausible slip in the oracle: a wrong FFT sign, index or twiddle
(brute-force DFT, Parseval), a wrong pair index or delay (travelling-cosine closed form, tau = 0),
a missing or wrong normalisation (scale invariance, OU closed form), a wrong half-plane weight
(full-plane Parseval identity), transposed k_x / k_y (non-square shapes in the bin count and the
closed forms).  The paper prints no worked numerical example, so there is no value to copy from it.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import nfs_synth as S


def brute_dft2(a):
    H, W = a.shape
    y = np.arange(H)
    x = np.arange(W)
    out = np.zeros((H, W), complex)
    for ky in range(H):
        for kx in range(W):
            ph = np.exp(-2j * np.pi * (ky * y[:, None] / H + kx * x[None, :] / W))
            out[ky, kx] = np.sum(a * ph)
    return out


@pytest.mark.parametrize("shape", [(8, 8), (6, 8), (12, 16), (9, 6)])
def test_fft_matches_brute_force_dft(oracle_lib, shape):
    rng = np.random.default_rng(1)
    a = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    ref = brute_dft2(a)
    got = oracle_lib.fft2(a)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.sqrt(np.sum(np.abs(ref) ** 2))


@pytest.mark.parametrize("shape", [(48, 32), (96, 72), (128, 128)])
def test_fft_parseval_and_library(oracle_lib, shape):
    rng = np.random.default_rng(2)
    a = rng.standard_normal(shape)
    F = oracle_lib.fft2(a)
    H, W = shape
    assert abs(np.sum(np.abs(F) ** 2) - H * W * np.sum(a * a)) <= 1e-12 * H * W * np.sum(a * a)
    # special case that reduces to a library routine: numpy's unscaled forward FFT
    assert np.max(np.abs(F - np.fft.fft2(a))) <= 1e-12 * np.sqrt(np.sum(np.abs(F) ** 2))


def test_tau_zero_and_identical_frames_are_exact_zero(oracle_lib):
    fr = S.uniform_frames(6, 12, 16, seed=3)
    r = oracle_lib.structure_function(fr, [0, 1, 2], 8, want_2d=True)
    assert np.all(r["D"][0] == 0.0) and np.all(r["D2d"][0] == 0.0)
    same = np.repeat(fr[:1], 5, axis=0)
    r2 = oracle_lib.structure_function(same, [1, 2, 4], 8, want_2d=True)
    assert np.all(r2["D"] == 0.0) and np.all(r2["D2d"] == 0.0)
    assert list(r2["pair_counts"]) == [4, 3, 1]


def test_dc_mode_of_normalised_differences_vanishes(oracle_lib):
    """Mean-normalised frames all sum to HW, so the difference's DC coefficient is 0 in exact
    arithmetic: in FP64 |Delta I(0)| <= 1e-9 HW (the reason the DC mode is left out of the bins)."""
    H, W = 24, 32
    fr = S.uniform_frames(12, H, W, seed=77)
    r = oracle_lib.structure_function(fr, [1, 3, 7], 8, want_2d=True)
    assert np.all(r["D2d"][:, 0, 0] <= (1e-9 * H * W) ** 2)
    assert np.all(r["D2d"][:, 0, 1:].max(axis=1) > 1e6 * r["D2d"][:, 0, 0])


def test_transpose_and_flip_invariance(oracle_lib):
    """Radial bins depend on |f| only, so transposing every frame (H x W -> W x H, which swaps the
    roles of k_x and k_y and of the half-plane axis) or mirroring it leaves every binned D unchanged;
    a swapped axis scale or half-plane weight would not."""
    fr = S.uniform_frames(10, 24, 32, seed=31)
    delays = [1, 2, 5]
    ref = oracle_lib.structure_function(fr, delays, 10)
    for g in (np.ascontiguousarray(fr.transpose(0, 2, 1)), np.ascontiguousarray(fr[:, :, ::-1]),
              np.ascontiguousarray(fr[:, ::-1, :])):
        r = oracle_lib.structure_function(g, delays, 10)
        np.testing.assert_array_equal(r["bin_counts"], ref["bin_counts"])
        np.testing.assert_allclose(r["D"], ref["D"], rtol=1e-11, atol=0)


def test_time_reversal_invariance(oracle_lib):
    fr = S.uniform_frames(9, 16, 12, seed=4)
    a = oracle_lib.structure_function(fr, [1, 2, 5], 6)["D"]
    b = oracle_lib.structure_function(fr[::-1].copy(), [1, 2, 5], 6)["D"]
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=0)


def test_intensity_scale_invariance(oracle_lib):
    fr = S.uniform_frames(7, 16, 16, seed=5, lo=1, hi=1000)
    sc = fr.copy()
    sc[2] *= 3
    sc[5] *= 7
    a = oracle_lib.structure_function(fr, [1, 3], 8)["D"]
    b = oracle_lib.structure_function(sc, [1, 3], 8)["D"]
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=0)


def test_fixed_image_offset_invariance(oracle_lib):
    rng = np.random.default_rng(6)
    n = 1.0 + 0.1 * rng.standard_normal((8, 12, 18))
    g = 5.0 * rng.standard_normal((12, 18))
    a = oracle_lib.structure_function(n, [1, 2, 3], 6, normalize=False)["D"]
    b = oracle_lib.structure_function(n + g[None], [1, 2, 3], 6, normalize=False)["D"]
    np.testing.assert_allclose(a, b, rtol=1e-10, atol=0)


def test_half_plane_weights_sum_like_full_plane(oracle_lib):
    """sum_k w_k D(k) over the half plane == (HW / (N - tau)) sum_t sum_x |Delta i|^2 (Parseval)."""
    fr = S.uniform_frames(6, 12, 16, seed=7)
    N, H, W = fr.shape
    r = oracle_lib.structure_function(fr, [1, 4], 4, want_2d=True)
    n = fr / fr.reshape(N, -1).mean(axis=1)[:, None, None]
    w = np.full(W // 2 + 1, 2.0)
    w[0] = w[-1] = 1.0
    for j, tau in enumerate([1, 4]):
        half = np.sum(r["D2d"][j] * w[None, :])
        full = H * W * np.mean([np.sum((n[t] - n[t + tau]) ** 2) for t in range(N - tau)])
        assert abs(half - full) <= 1e-12 * full


def test_fft_linearity_route_matches_real_space_route(oracle_lib):
    """Transforming each frame once and differencing spectra (the paper's speed-up) gives the same D."""
    fr = S.uniform_frames(10, 24, 18, seed=8)
    N, H, W = fr.shape
    delays = [1, 2, 7]
    r = oracle_lib.structure_function(fr, delays, 6, want_2d=True)
    n = fr / fr.reshape(N, -1).mean(axis=1)[:, None, None]
    F = np.fft.rfft2(n)
    for j, tau in enumerate(delays):
        ref = np.mean([np.abs(F[t] - F[t + tau]) ** 2 for t in range(N - tau)], axis=0)
        np.testing.assert_allclose(r["D2d"][j], ref, rtol=1e-12, atol=1e-12 * ref.max())


def _frac_bin(kx, ky, H, W, nq):
    """Bin by exact rational comparison of 2 nq |f| with the integers (independent of the lcm form)."""
    kys = ky if ky <= H // 2 else ky - H
    f2 = Fraction(kx * kx, W * W) + Fraction(kys * kys, H * H)  # |f|^2 in (cycles/px)^2
    x2 = 4 * nq * nq * f2  # (2 nq |f|)^2
    b = 0
    while Fraction((b + 1) ** 2) <= x2:
        b += 1
    return b


@pytest.mark.parametrize("H,W,nq", [(6, 8, 3), (12, 16, 8), (64, 64, 32), (128, 128, 64), (48, 64, 24),
                                    (24, 32, 40)])
def test_bin_table_matches_exact_brute_force(oracle_lib, H, W, nq):
    b, c, q = oracle_lib.bins(H, W, nq)
    cnt = np.zeros(nq, np.int64)
    qs = np.zeros(nq)
    for ky in range(H):
        for kx in range(W // 2 + 1):
            bb = _frac_bin(kx, ky, H, W, nq)
            keep = bb < nq and (kx, ky) != (0, 0)
            assert b[ky, kx] == (bb if keep else -1), (ky, kx)
            if keep:
                w = 1 if kx in (0, W // 2) else 2
                cnt[bb] += w
                kys = ky if ky <= H // 2 else ky - H
                qs[bb] += w * 2 * np.pi * math.hypot(kx / W, kys / H)
    np.testing.assert_array_equal(c, cnt)
    nz = cnt > 0
    np.testing.assert_allclose(q[nz], qs[nz] / cnt[nz], rtol=1e-13)
    # bins span 0 <= |f| < 0.5 cycles/px, so the weighted half plane counts every full-plane mode
    # with 0 < |f| < 0.5 exactly once
    fy = np.fft.fftfreq(H)[:, None]
    fx = np.fft.fftfreq(W)[None, :]
    f2 = fy ** 2 + fx ** 2
    assert c.sum() == int(np.sum((f2 < 0.25) & (f2 > 0)))


def test_bin_table_exact_beyond_64_bits(oracle_lib):
    """4 n_q^2 r2 beyond 64 bits (H = 486, W = 2048: lcm 497,664; n_q = 8000): every bin is the
    largest b with (b L)^2 <= 4 n_q^2 r2, checked in Python integers."""
    H, W, nq = 486, 2048, 8000
    b, c, _ = oracle_lib.bins(H, W, nq)
    L = H * W // math.gcd(H, W)
    assert 4 * nq * nq * ((W // 2 * (L // W)) ** 2 + (H // 2 * (L // H)) ** 2) >= 2 ** 64
    cnt = np.zeros(nq, np.int64)
    for ky in range(H):
        kys = ky if ky <= H // 2 else ky - H
        n = kys * (L // H)
        for kx in range(W // 2 + 1):
            m = kx * (L // W)
            bb = math.isqrt(4 * nq * nq * (m * m + n * n)) // L
            keep = bb < nq and (kx, ky) != (0, 0)
            if b[ky, kx] != (bb if keep else -1):
                raise AssertionError((ky, kx, int(b[ky, kx]), bb))
            if keep:
                cnt[bb] += 1 if kx in (0, W // 2) else 2
    np.testing.assert_array_equal(c, cnt)


def test_travelling_cosine_closed_form(oracle_lib):
    """n_t = 1 + eps cos(2 pi k0.x + omega t): |Delta I(k0)|^2 = (eps HW / 2)^2 2 (1 - cos(omega tau))."""
    H, W, kx0, ky0, eps, om = 24, 32, 3, 5, 0.2, 0.37
    N = 12
    n = S.travelling_cosine_frames(N, H, W, kx0, ky0, eps, om)
    delays = [0, 1, 2, 5, 11]
    nq = 16
    r = oracle_lib.structure_function(n, delays, nq, normalize=False, want_2d=True)
    amp = (eps * H * W / 2.0) ** 2
    b0 = _frac_bin(kx0, ky0, H, W, nq)
    for j, tau in enumerate(delays):
        exp = amp * 2.0 * (1.0 - math.cos(om * tau))
        D2 = r["D2d"][j]
        assert abs(D2[ky0, kx0] - exp) <= 1e-12 * amp
        mask = np.ones_like(D2, bool)
        mask[ky0, kx0] = False
        assert np.max(np.abs(D2[mask])) <= 1e-12 * amp
        Db = np.zeros(nq)
        Db[b0] = 2.0 * exp / r["bin_counts"][b0]
        np.testing.assert_allclose(r["D"][j], Db, rtol=1e-12, atol=1e-12 * amp / r["bin_counts"][b0])
    assert list(r["pair_counts"]) == [N - t for t in delays]


def test_dark_frames_closed_form(oracle_lib):
    """Dark frames (spatial mean 0) normalise to the zero image.  With frames c_t (1 + eps cos(2 pi
    k0.x + omega t)) (any scale c_t > 0) and dark frames in between: a pair of two lit frames gives
    (eps HW / 2)^2 2 (1 - cos(omega tau)) at k0 and 0 at DC; a pair with one dark frame gives
    (eps HW / 2)^2 at k0 and (HW)^2 at DC; every other mode 0."""
    H, W, kx0, ky0, eps, om = 24, 32, 3, 5, 0.2, 0.37
    N = 12
    dark = {0, 4, 5}
    n = S.travelling_cosine_frames(N, H, W, kx0, ky0, eps, om)
    scale = 1.0 + np.arange(N)
    frames = n * scale[:, None, None]
    for t in dark:
        frames[t] = 0.0
    delays = [0, 1, 2, 5, 11]
    r = oracle_lib.structure_function(frames, delays, 16, normalize=True, want_2d=True)
    amp = (eps * H * W / 2.0) ** 2
    for j, tau in enumerate(delays):
        pairs = [(t, t + tau) for t in range(N - tau)]
        lit = sum(1 for a, b in pairs if a not in dark and b not in dark)
        one = sum(1 for a, b in pairs if (a in dark) != (b in dark))
        D2 = r["D2d"][j]
        exp_k0 = (lit * amp * 2.0 * (1.0 - math.cos(om * tau)) + one * amp) / len(pairs)
        exp_dc = one * float(H * W) ** 2 / len(pairs)
        assert abs(D2[ky0, kx0] - exp_k0) <= 1e-12 * amp
        assert abs(D2[0, 0] - exp_dc) <= 1e-12 * float(H * W) ** 2
        mask = np.ones_like(D2, bool)
        mask[ky0, kx0] = False
        mask[0, 0] = False
        assert np.max(np.abs(D2[mask])) <= 1e-12 * amp
    # uint16 frames: the one-mode route agrees with the full oracle when frames are dark
    u = np.clip(np.rint(frames * 1000.0), 0, 4095).astype(np.uint16)
    ru = oracle_lib.structure_function(u, [1, 4], 16, want_2d=True)
    for j, tau in enumerate([1, 4]):
        for kx, ky in ((kx0, ky0), (0, 1), (W // 2, 7)):
            v = oracle_lib.mode_power(u, kx, ky, tau)
            assert abs(v - ru["D2d"][j][ky, kx]) <= 1e-12 * max(abs(v), amp)


def test_ou_statistical_closed_form(oracle_lib):
    """Eq. 1 with f = exp(-Gamma tau) and no noise: E D(k, tau) = 2 eps^2 s^2 (HW)^2 S_k (1 - e^{-Gamma_k tau}).

    Flat illumination, FP64 frames P0 (1 + eps phi_t) built from OU Fourier modes with known
    Gamma = Dc q^2; s^2 = 1 / sum(S) over the full plane.  Statistical, so the tolerance is loose.
    """
    H = W = 64
    nq = 32
    N = 600
    src = S.OUFrameSource(H, W, Dc=2.0, gamma0=0.02, flat=True, shot_noise=False, seed=11)
    phi = src.fields(N).numpy()
    frames = 2000.0 * (1.0 + src.eps * phi)
    delays = [1, 3, 10]
    r = oracle_lib.structure_function(frames, delays, nq)
    Sk = src.S.numpy()
    G = src.gamma.numpy()
    s2 = src.field_scale ** 2
    b, c, _ = oracle_lib.bins(H, W, nq)
    w = np.full(W // 2 + 1, 2.0)
    w[0] = w[-1] = 1.0
    for j, tau in enumerate(delays):
        Dk = 2 * src.eps ** 2 * s2 * (H * W) ** 2 * Sk * (1 - np.exp(-G * tau))
        exp = np.array([np.sum((w[None, :] * Dk)[b == q]) / c[q] if c[q] else 0.0 for q in range(nq)])
        sel = slice(3, 20)  # bins with enough modes and S well above rounding
        rel = r["D"][j, sel] / exp[sel] - 1.0
        assert np.abs(np.mean(rel)) < 0.03, rel
        assert np.max(np.abs(rel)) < 0.15, rel


def test_mode_power_matches_full_transform(oracle_lib):
    fr = S.uniform_frames(8, 16, 24, seed=9)
    r = oracle_lib.structure_function(fr, [2], 4, want_2d=True)
    for kx, ky in [(0, 1), (3, 5), (12, 15), (7, 0)]:
        v = oracle_lib.mode_power(fr, kx, ky, 2)
        assert abs(v - r["D2d"][0, ky, kx]) <= 1e-11 * r["D2d"][0].max()


def test_all_delays_enumerate_every_pair(oracle_lib):
    """All N-1 delays visit N(N-1)/2 pairs (the processing paragraph's count of differences)."""
    fr = S.uniform_frames(11, 8, 8, seed=10)
    r = oracle_lib.structure_function(fr, list(range(1, 11)), 4)
    assert int(r["pair_counts"].sum()) == 11 * 10 // 2


def test_log_delay_rule():
    d2 = S.log_delays(1, 500, 100)
    assert d2[:68] == list(range(1, 69)) and d2[68:70] == [71, 76] and d2[-2:] == [470, 500]
    assert sum(1000 - t for t in d2) == 90538
    d3 = S.log_delays(1, 2000, 200)
    assert d3[:128] == list(range(1, 129)) and d3[128] == 133 and d3[-2:] == [1925, 2000]
    assert sum(4000 - t for t in d3) == 741785
    assert len(set(d3)) == 200 and all(b > a for a, b in zip(d3, d3[1:]))
