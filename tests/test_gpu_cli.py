"""The command-line front end on a GPU: its result file equals the library's result for the same
frames (it only reads the file and marshals arguments)."""
import numpy as np
import pytest

import nfs_synth as S
import paper_1209_3362_gb300 as P
from paper_1209_3362_gb300.__main__ import main

pytestmark = pytest.mark.gpu


def test_cli_matches_the_library(tmp_path):
    P.build()
    fr = S.OUFrameSource(64, 96, 1.0, seed=9).frames_numpy(300)
    np.save(tmp_path / "f.npy", fr)
    delays = S.log_delays(1, 100, 20)
    main([str(tmp_path / "f.npy"), "--delays", "log:1:100:20", "--bins", "32", "--chunk", "77",
          "--out", str(tmp_path / "r.npz")])
    r = np.load(tmp_path / "r.npz")
    with P.NFS(64, 96, delays, 32) as ctx:
        ctx.push_frames(fr)
        ref = ctx.structure_function()
    np.testing.assert_array_equal(r["tau"], delays)
    np.testing.assert_array_equal(r["D"], ref["D"])
    np.testing.assert_array_equal(r["pair_counts"], ref["pair_counts"])
    main([str(tmp_path / "f.npy"), "--delays", "log:1:100:20", "--bins", "16", "--roi", "0", "0", "32", "48",
          "--roi", "16", "40", "48", "48", "--out", str(tmp_path / "roi.npz")])
    q = np.load(tmp_path / "roi.npz")
    with P.NFS(32, 48, delays, 16) as ctx:
        ctx.push_frames(np.ascontiguousarray(fr[:, 0:32, 0:48]))
        ref0 = ctx.structure_function()
    np.testing.assert_array_equal(q["roi0_D"], ref0["D"])
    assert q["roi1_D"].shape == (20, 16)
