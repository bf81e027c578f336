"""Regions of interest (nfs_roi_*): windows of one camera sequence, each analysed as a sequence of
its own (spatially resolved analysis).  Every window's result must equal, bit for bit, a single
context fed the cropped frames, and match the FP64 oracle on the cropped frames."""
import numpy as np
import pytest
import torch

import nfs_synth as S
import paper_1209_3362_gb300 as P

pytestmark = pytest.mark.gpu

TOL_F32 = 2e-5
H, W, N = 192, 256, 600          # 600 frames: more than one 512-frame block and 64-frame crop group
ROIS = [(0, 0, 96, 128),          # (y0, x0, h, w)
        (96, 128, 96, 128),
        (32, 40, 64, 64),         # overlaps the first window
        (100, 2, 48, 96),
        (0, 0, 192, 256)]         # the whole frame
ORACLE_ROIS = (0, 2, 3)


def rel_err(got, ref):
    m = (ref["bin_counts"][None, :] > 0) & (ref["pair_counts"][:, None] > 0) & (ref["D"] != 0)
    assert np.all(got["D"][~m & (ref["D"] == 0)] == 0.0)
    return float(np.max(np.abs(got["D"][m] - ref["D"][m]) / np.abs(ref["D"][m])))


def crop(frames, r):
    y0, x0, h, w = r
    return np.ascontiguousarray(frames[:, y0:y0 + h, x0:x0 + w])


@pytest.fixture(scope="module")
def case(oracle_lib):
    P.build()
    frames = S.OUFrameSource(H, W, 0.8, seed=1209).frames_numpy(N)
    delays = S.log_delays(1, 250, 40)
    nqs = [min(h, w) // 2 for _, _, h, w in ROIS]
    singles = []
    for r, nq in zip(ROIS, nqs):
        with P.NFS(r[2], r[3], delays, nq) as ctx:
            ctx.push_frames(crop(frames, r))
            singles.append(ctx.structure_function())
    refs = {i: oracle_lib.structure_function(crop(frames, ROIS[i]), delays, nqs[i]) for i in ORACLE_ROIS}
    return frames, delays, nqs, singles, refs


def check(got, case):
    frames, delays, nqs, singles, refs = case
    for i in range(len(ROIS)):
        np.testing.assert_array_equal(got[i]["D"], singles[i]["D"])
        np.testing.assert_array_equal(got[i]["bin_counts"], singles[i]["bin_counts"])
        np.testing.assert_array_equal(got[i]["pair_counts"], singles[i]["pair_counts"])
    for i, ref in refs.items():
        np.testing.assert_array_equal(got[i]["bin_counts"], ref["bin_counts"])
        np.testing.assert_array_equal(got[i]["pair_counts"], ref["pair_counts"])
        assert rel_err(got[i], ref) <= TOL_F32, i


def test_roi_host_pushes_in_uneven_pieces(case):
    frames, delays, nqs = case[:3]
    with P.NFSRoi(H, W, ROIS, delays, nqs) as b:
        for lo, hi in ((0, 37), (37, 137), (137, 600)):
            b.push_frames(frames[lo:hi])
        got = [b.structure_function(i) for i in range(len(ROIS))]
    check(got, case)


def test_roi_device_push_and_reset(case):
    frames, delays, nqs = case[:3]
    dev = torch.from_numpy(frames.view(np.int16)).cuda()
    with P.NFSRoi(H, W, ROIS, delays, nqs) as b:
        b.push_frames_device(dev[:100])  # a partial run first, then reset
        b.synchronize()
        b.reset()
        b.push_frames_device(dev)
        got = [b.structure_function(i) for i in range(len(ROIS))]
        # the crop adds one launch per 64-frame group to the members' launches
        assert b.launch_count > 0
    check(got, case)


def test_roi_pinned_host_buffer(case):
    frames, delays, nqs = case[:3]
    pinned = torch.from_numpy(frames.view(np.int16)).pin_memory()
    with P.NFSRoi(H, W, ROIS[:2], delays, nqs[:2]) as b:
        b.push_frames(pinned.numpy().view(np.uint16))
        got = [b.structure_function(i) for i in range(2)]
    for i in range(2):
        np.testing.assert_array_equal(got[i]["D"], case[3][i]["D"])
