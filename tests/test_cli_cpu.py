"""The command-line front end on the host: delay specifications, frame files, and no CPU
fallback (without a GPU the analysis raises)."""
import numpy as np
import pytest

import nfs_synth as S
import paper_1209_3362_gb300 as P
from paper_1209_3362_gb300.__main__ import load_frames, main, parse_delays


def test_delay_specs():
    assert parse_delays("log:1:2000:200") == S.log_delays(1, 2000, 200)
    assert parse_delays("log:1:500:100") == S.log_delays(1, 500, 100)
    assert parse_delays("range:3:7") == [3, 4, 5, 6, 7]
    assert parse_delays("1, 2,5") == [1, 2, 5]
    with pytest.raises(ValueError):
        parse_delays("5,3")


def test_frame_files(tmp_path):
    fr = S.uniform_frames(4, 6, 8, seed=1)
    np.save(tmp_path / "f.npy", fr)
    fr.tofile(tmp_path / "f.raw")
    np.testing.assert_array_equal(load_frames(str(tmp_path / "f.npy")), fr)
    np.testing.assert_array_equal(load_frames(str(tmp_path / "f.raw"), (6, 8)), fr)
    with pytest.raises(ValueError):
        load_frames(str(tmp_path / "f.raw"), (5, 8))
    np.save(tmp_path / "g.npy", fr.astype(np.int32))
    with pytest.raises(ValueError):
        load_frames(str(tmp_path / "g.npy"))


def test_no_cpu_fallback(tmp_path):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    P.build()
    np.save(tmp_path / "f.npy", S.uniform_frames(4, 8, 8, seed=2))
    with pytest.raises(P.NFSError):
        main([str(tmp_path / "f.npy"), "--delays", "1,2", "--bins", "4", "--out", str(tmp_path / "r.npz")])
