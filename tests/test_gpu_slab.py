"""Mode slabs on one GPU: the slab contexts of one frame sequence add up to the whole context (the
split of the delay update and of the column transforms by mode is exact; only the FP64 sum of the
bin shares rounds differently), for two and three slabs, host and device pushes, and the 2-D
exports of the slabs add up to the whole export mode by mode."""
import numpy as np
import pytest

import nfs_synth as S

torch = pytest.importorskip("torch")


@pytest.mark.gpu
@pytest.mark.parametrize("H,W,n_slabs", [(96, 128, 2), (96, 128, 3), (256, 256, 5), (384, 512, 2)])
def test_slabs_add_up_to_the_whole_context(H, W, n_slabs):
    import paper_1209_3362_gb300 as P
    P.build()
    fr = S.OUFrameSource(H, W, 1.1, seed=H + n_slabs).frames_numpy(640)
    delays, nq = [1, 2, 3, 4, 5, 17, 100, 300, 530], 32
    with P.NFS(H, W, delays, nq) as whole:
        whole.set_option(P.OPT_MODES, 1)  # every mode: the 2-D exports compared below
        whole.push_frames(fr)
        ref = whole.structure_function()
        ex_ref = whole.export_spectrum(6)
    parts, exports = [], []
    dev = torch.from_numpy(fr.view(np.int16)).cuda()
    for s in range(n_slabs):
        with P.NFS(H, W, delays, nq, slab=s, n_slabs=n_slabs) as c:
            first, n = P.slab_range(H, W, s, n_slabs)
            assert (c.get_option(P.OPT_SLAB_FIRST_MODE), c.get_option(P.OPT_SLAB_MODES)) == (first, n)
            c.set_option(P.OPT_MODES, 1)
            if s % 2:
                c.push_frames(fr[:333])
                c.push_frames(fr[333:])
            else:
                c.push_frames_device(dev)
            parts.append(c.structure_function())
            exports.append(c.export_spectrum(6))
    red = P.reduce_slabs(parts)
    assert np.array_equal(red["bin_counts"], ref["bin_counts"]) and np.array_equal(red["pair_counts"], ref["pair_counts"])
    assert np.array_equal(red["q_mean"], ref["q_mean"])
    m = ref["D"] != 0
    assert np.all(red["D"][~m] == 0)
    assert np.max(np.abs(red["D"][m] - ref["D"][m]) / np.abs(ref["D"][m])) <= 1e-12
    # every mode belongs to exactly one slab: the exports add up exactly
    assert np.array_equal(np.sum(exports, axis=0), ex_ref)
