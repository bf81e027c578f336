"""Failure detection without a GPU fault: a copy group that is never issued makes a consumer's
bounded wait in the fused delay kernel run out; the kernel records where, every other CTA stops
waiting at once, and the host returns NFS_ETIMEOUT (sticky) while the GPU stays usable."""
import numpy as np
import pytest
import torch

import nfs_synth as S
import paper_1209_3362_gb300 as P

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_is_reported(oracle_lib):
    assert torch.cuda.is_available()
    fr = S.uniform_frames(300, 64, 64, seed=71)
    delays = list(range(1, 21)) + [100]
    with P.NFS(64, 64, delays, 16) as ctx:
        ctx.set_option(P.OPT_TEST_STALL_GROUP, 1)  # stage 0's group never arrives
        ctx.push_frames(fr)
        with pytest.raises(P.NFSError) as e:
            ctx.structure_function()
        assert e.value.status == P.NFS_ETIMEOUT
        msg = str(e.value)
        # the first waiter to give up is a consumer waiting for the copy group (kind 1) or the
        # writer waiting for the batch those consumers could not finish (kind 2); every consumer
        # warp is recorded as stuck after step 1 (the block's own frames) with no batch handed over
        assert ("kind 1" in msg or "kind 2" in msg) and "per warp: " + " ".join(["1/0"] * 16) in msg, msg
        with pytest.raises(P.NFSError) as e2:  # sticky
            ctx.push_frames(fr[:1])
        assert e2.value.status == P.NFS_ETIMEOUT
    # the device is healthy: a fresh context gives the right answer
    ref = oracle_lib.structure_function(fr[:60], delays, 16)
    with P.NFS(64, 64, delays, 16) as ctx:
        ctx.push_frames(fr[:60])
        got = ctx.structure_function()
    m = (ref["bin_counts"][None, :] > 0) & (ref["pair_counts"][:, None] > 0)
    assert np.max(np.abs(got["D"][m] - ref["D"][m]) / ref["D"][m]) <= 2e-5
