"""The seeded input generators (no analysis arithmetic): reproducible, 12-bit, with the beam and
workload geometry they document."""
import numpy as np

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
    """Mean counts follow the Gaussian beam: peak P0 = 2000 at the centre, sigma = 40 px at 128^2."""
    fr = S.OUFrameSource(128, 128, 0.5, seed=11).frames_numpy(40).astype(np.float64)
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
