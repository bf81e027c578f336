"""The counter-based frame generator gives the same frames on the CPU and on the GPU (the full-size
oracle fixtures are computed from CPU frames and checked against GPU-generated ones)."""
import numpy as np
import pytest

import nfs_synth as S

torch = pytest.importorskip("torch")


@pytest.mark.gpu
@pytest.mark.parametrize("H,W,Dc,g0,n,seed", [(128, 128, 0.5, 0.0, 48, 12093363), (96, 384, 2.0, 0.01, 20, 5),
                                              (2048, 2048, 1.0, 0.01, 3, 12093365)])
def test_frames_equal_on_cpu_and_gpu(H, W, Dc, g0, n, seed):
    a = S.OUFrameSource(H, W, Dc, g0, seed=seed).frames_numpy(n)
    b = S.OUFrameSource(H, W, Dc, g0, seed=seed, device="cuda").frames_numpy(n)
    diff = int(np.count_nonzero(a != b))
    # draws are integer-exact; FP64 rounding differs between devices only in the last place, which
    # moves a count only when a rate sits within ~1e-13 of a rounding edge
    assert diff <= 1, f"{diff} of {a.size} pixels differ"
    assert np.array_equal(S.frame_checksums(a) if diff == 0 else S.frame_checksums(b), S.frame_checksums(b))
