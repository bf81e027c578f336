"""Timeline tracing (NFS_OPT_TIMING = 3, nfs_get_timeline): every copy and launch of a host push
is recorded once, with start <= end, and the stage totals agree with nfs_get_timings."""
import numpy as np
import pytest

import nfs_synth as S

torch = pytest.importorskip("torch")


@pytest.mark.gpu
def test_timeline_of_a_host_push():
    import paper_1209_3362_gb300 as P
    P.build()
    fr = S.OUFrameSource(64, 96, 1.0, seed=23).frames_numpy(700)
    with P.NFS(64, 96, [1, 2, 3, 50, 400], 16) as c:
        c.set_option(P.OPT_TIMING, 3)
        c.reset_timings()
        c.push_frames(fr[:300])
        c.push_frames(fr[300:])
        c.structure_function()
        tl = c.timeline()
        tot = c.timings()
        assert len(tl) > 0 and all(b >= a for _, a, b in tl)
        for st in P.STAGES:
            ent = [(a, b) for s, a, b in tl if s == st]
            assert len(ent) == tot[st][1], st
            assert abs(sum(b - a for a, b in ent) - tot[st][0]) <= 1e-3 * max(1.0, tot[st][0]), st
        # two blocks of 512 frames: the first is complete at frame 512, the rest flushes at the end
        assert sum(1 for s, _, _ in tl if s == "delay") == 2
        assert min(a for _, a, _ in tl) >= -1e-3
        c.reset_timings()
        assert c.timeline() == []
