"""The seeded input generators (no analysis arithmetic): reproducible, 12-bit, with the beam and
workload geometry they document."""
import numpy as np
import pytest
import torch

import nfs_synth as S


def test_frames_are_seeded_and_12_bit():
    a = S.OUFrameSource(64, 96, 0.8, seed=5).frames_numpy(6)
    b = S.OUFrameSource(64, 96, 0.8, seed=5).frames_numpy(6)
    c = S.OUFrameSource(64, 96, 0.8, seed=6).frames_numpy(6)
    assert a.dtype == np.uint16 and a.shape == (6, 64, 96)
    np.testing.assert_array_equal(a, b)
    assert not np.array_equal(a, c)
    assert a.max() <= 4095


def test_beam_profile_peak_and_width():
    """Mean counts follow the Gaussian beam: peak P0 = 2000 at the centre, sigma = 40 px at 128^2
    (the fluctuating field is switched off, eps = 0: its slow low-q modes would move the mean of a
    few frames by several per cent)."""
    fr = S.OUFrameSource(128, 128, 0.5, eps=0.0, seed=11).frames_numpy(40).astype(np.float64)
    m = fr.mean(axis=0)
    assert abs(m[62:66, 62:66].mean() / 2000.0 - 1.0) < 0.05
    sigma = S.beam_sigma(128, 128)
    assert sigma == 40.0
    y = m[64, :]
    # at one sigma from the centre the profile is exp(-1/2) of the peak
    assert abs(y[64 + 40] / y[64] - np.exp(-0.5)) < 0.08


def test_uniform_frames_range():
    u = S.uniform_frames(5, 8, 10, seed=3, lo=7, hi=9)
    assert u.min() >= 7 and u.max() <= 9 and u.dtype == np.uint16


def test_workload_geometry():
    w = S.ROI_WORKLOADS["roi2048"]
    rois = w.rois()
    assert len(rois) == w.grid[0] * w.grid[1]
    cover = np.zeros((w.H, w.W), np.int32)
    for y0, x0, h, wd in rois:
        cover[y0:y0 + h, x0:x0 + wd] += 1
    assert np.all(cover == 1)  # the windows tile the frame exactly
    r = S.RAGGED_WORKLOADS["ragged48"]
    m1, m2 = r.members(), r.members()
    assert m1 == m2 and len(m1) == r.n_seq
    assert all(len(m[3]) == 64 and m[3][-1] == r.N // 2 and m[4] == min(m[0], m[1]) // 2 for m in m1)
    for w in S.WORKLOADS.values():
        assert all(b > a for a, b in zip(w.delays, w.delays[1:])) and w.delays[-1] < w.N


# Known-answer vectors of Philox4x32-10 published with the Random123 library (Salmon et al., SC 2011):
# (counter words, key words) -> output words.
PHILOX_KAT = [
    ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
    ((0xFFFFFFFF,) * 4, (0xFFFFFFFF, 0xFFFFFFFF), (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
    ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
     (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
]


@pytest.mark.parametrize("ctr,key,out", PHILOX_KAT)
def test_philox_known_answers(ctr, key, out):
    got = S.philox4x32(*ctr, *key)
    assert tuple(int(v) for v in got) == out


def test_philox_is_counter_based():
    """Element i of a batch equals the single draw of counter i (chunking, broadcasting and batch
    sizes do not change the stream), and every output word stays a uint32."""
    n = (1 << 18) + 77  # crosses the CPU chunk size
    big = S.philox4x32(torch.arange(n), 5, 1, 9, 3, 4)
    for i in (0, 1, (1 << 18) - 1, 1 << 18, n - 1):
        one = S.philox4x32(i, 5, 1, 9, 3, 4)
        assert all(int(b[i]) == int(o) for b, o in zip(big, one))
    assert all(int(w.min()) >= 0 and int(w.max()) < (1 << 32) for w in big)
    # the low bits are balanced
    bits = (big[0][:, None] >> torch.arange(32)) & 1
    assert torch.all(torch.abs(bits.double().mean(0) - 0.5) < 0.005)


def test_complex_normals_moments():
    z = S.complex_normals(400000, 3, S.STREAM_STEP, (7, 8), torch.float64, "cpu").numpy()
    for part in (z.real, z.imag):
        assert abs(part.mean()) < 0.005 and abs(part.var() - 0.5) < 0.005
    assert abs(np.mean(z.real * z.imag)) < 0.005
    assert abs(np.mean(np.abs(z) ** 4) - 2.0) < 0.03  # E|z|^4 = 2 for CN(0, 1)


@pytest.mark.parametrize("lam", [0.7, 3.2, 9.9, 10.0, 37.5, 154.0, 2000.0])
def test_poisson_counts_match_the_pmf(lam):
    """Both samplers (inversion below 10, PTRS from 10) against the Poisson pmf: chi-square per
    degree of freedom over cells with >= 20 expected counts, and the mean and variance."""
    from scipy import stats
    k = S.poisson_counts(torch.full((2, 256, 512), lam, dtype=torch.float64), 11, (123, 4)).numpy().ravel()
    assert np.all(k == np.floor(k)) and k.min() >= 0
    vals, cnt = np.unique(k.astype(np.int64), return_counts=True)
    exp = stats.poisson.pmf(vals, lam) * k.size
    m = exp >= 20
    chi2 = float(np.sum((cnt[m] - exp[m]) ** 2 / exp[m]))
    dof = int(m.sum()) - 1
    assert stats.chi2.sf(chi2, dof) > 1e-4, (chi2, dof)
    se = np.sqrt(lam / k.size)
    assert abs(k.mean() - lam) < 5 * se
    assert abs(k.var() / lam - 1.0) < 0.02


def test_frames_do_not_depend_on_the_batch_split():
    """Counter-based draws: frames produced 6 at once or as 2 + 4 are the same frames."""
    a = S.OUFrameSource(48, 64, 1.3, seed=19).frames_numpy(6)
    src = S.OUFrameSource(48, 64, 1.3, seed=19)
    b = np.concatenate([src.frames_numpy(2), src.frames_numpy(4)])
    assert np.array_equal(a, b)
    cs = S.frame_checksums(a)
    assert cs.shape == (6, 2) and np.array_equal(cs, S.frame_checksums(torch.from_numpy(b.view(np.int16))))
