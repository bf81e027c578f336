"""Host pushes: the SMs' copy kernel (NFS_OPT_H2D = 0, the default), which also takes the frames'
exact sums on the way, and the copy engines (NFS_OPT_H2D = 1) followed by the sum kernel give the
same sums and the same bytes, so the structure functions are bit-identical; a pinned source that
is not 16-byte aligned falls back to the copy engines with the same result."""
import numpy as np
import pytest

import nfs_synth as S

torch = pytest.importorskip("torch")

H, W = 64, 96
DELAYS = [1, 2, 3, 17, 300]


def _run(P, frames, h2d, split=(0, 300, 700)):
    """Result and the launches of the mean stage (sum kernels and the one reference image)."""
    with P.NFS(H, W, DELAYS, 16) as c:
        c.set_option(P.OPT_H2D, h2d)
        assert c.get_option(P.OPT_H2D) == h2d
        c.set_option(P.OPT_TIMING, 1)
        for a, b in zip(split[:-1], split[1:]):
            c.push_frames(frames[a:b])
        r = c.structure_function()
        return r, c.timings()["mean"][1]


@pytest.mark.gpu
def test_sm_reads_and_copy_engines_are_bit_identical():
    import paper_1209_3362_gb300 as P
    P.build()
    fr = S.OUFrameSource(H, W, 1.0, seed=31).frames_numpy(700)
    pinned = torch.from_numpy(fr.view(np.int16)).pin_memory()
    r_sm, n_sm = _run(P, pinned, 0)
    r_ce, n_ce = _run(P, pinned, 1)
    np.testing.assert_array_equal(r_sm["D"], r_ce["D"])
    np.testing.assert_array_equal(r_sm["pair_counts"], r_ce["pair_counts"])
    # the SM copy kernel takes the sums itself: the mean stage is the reference image alone, while
    # the copy engines' chunks each need a sum launch
    assert n_sm == 1 and n_ce > 1
    # pageable sources pass through the library's own pinned chunks, then the same kernel
    r_pg, n_pg = _run(P, fr, 0)
    np.testing.assert_array_equal(r_pg["D"], r_ce["D"])
    assert n_pg == n_sm


@pytest.mark.gpu
def test_unaligned_pinned_source_falls_back_to_the_copy_engines():
    import paper_1209_3362_gb300 as P
    P.build()
    fr = S.OUFrameSource(H, W, 1.0, seed=37).frames_numpy(700)
    buf = torch.empty(700 * H * W + 1, dtype=torch.int16).pin_memory()
    buf[1:] = torch.from_numpy(fr.view(np.int16).reshape(-1))
    view = buf[1:].view(700, H, W)  # 2 bytes past a 16-byte boundary
    assert view.data_ptr() % 16 == 2
    r_un, n_un = _run(P, view, 0)
    r_ce, n_ce = _run(P, torch.from_numpy(fr.view(np.int16)).pin_memory(), 1)
    np.testing.assert_array_equal(r_un["D"], r_ce["D"])
    assert n_un == n_ce
    with P.NFS(H, W, DELAYS, 16) as c:
        with pytest.raises(P.NFSError):
            c.set_option(P.OPT_H2D, 2)


@pytest.mark.gpu
def test_region_of_interest_push_from_pinned_memory():
    import paper_1209_3362_gb300 as P
    P.build()
    fr = S.OUFrameSource(H, W, 1.0, seed=41).frames_numpy(120)
    pinned = torch.from_numpy(fr.view(np.int16)).pin_memory()
    out = []
    for src in (pinned, fr):
        with P.NFSRoi(H, W, [(0, 0, 32, 32), (8, 40, 48, 48)], [1, 2, 5], [8, 12]) as r:
            r.push_frames(src)
            out.append([r.structure_function(i)["D"] for i in range(2)])
    for a, b in zip(*out):
        np.testing.assert_array_equal(a, b)
