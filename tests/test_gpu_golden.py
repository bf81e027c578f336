"""Full-size parity against stored FP64 oracle values (Eq. 1 averaged over every pair at each delay,
azimuthal average of Fig. 1e,f): the 1024x1024 sequence (1000 frames, all 100 log delays 1..500,
512 bins) and the 2048x2048 sequence (4000 frames, 200 log delays 1..2000, 1024 bins; every 10th
delay and the last one are stored).  tests/golden/make_golden.py wrote the fixtures on the CPU from
the workloads' counter-based frames by calling only the oracle; here the same frames are generated
on the GPU, checked against the fixture's per-frame checksums, pushed from page-locked host memory
through nfs_push_frames, and the binned D is compared element by element at the FP32 path's 2e-5
with every count exact."""
import os

import numpy as np
import pytest

import nfs_synth as S

torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))
TOL_F32 = 2e-5


def fixture(name):
    p = os.path.join(HERE, "golden", f"{name}_oracle.npz")
    if not os.path.exists(p):
        pytest.fail(f"missing oracle fixture {p} (tests/golden/make_golden.py {name})")
    return np.load(p)


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["ddm1024", "ddm2048"])
def test_full_size_sequence_matches_the_stored_oracle(name):
    import paper_1209_3362_gb300 as P
    P.build()
    w = S.WORKLOADS[name]
    z = fixture(name)
    assert (int(z["N"]), int(z["H"]), int(z["W"]), int(z["seed"])) == (w.N, w.H, w.W, w.seed)
    assert np.array_equal(z["delays_all"], np.asarray(w.delays)) and int(z["n_qbins"]) == w.n_qbins
    src = S.workload_source(w, device="cuda")
    batch = 32
    host = torch.empty((batch, w.H, w.W), dtype=torch.int16, pin_memory=True)
    sums = np.zeros((w.N, 2), np.int64)
    with P.NFS(w.H, w.W, w.delays, w.n_qbins) as ctx:
        for o in range(0, w.N, batch):
            n = min(batch, w.N - o)
            f = src.next_frames(n)
            sums[o:o + n] = S.frame_checksums(f)
            host[:n].copy_(f)
            ctx.push_frames(host[:n])
        r = ctx.structure_function()
    # the frames are the fixture's (a count moves only if a rate sits within ~1e-13 of a rounding
    # edge; such a one-count change moves D by ~1e-8, far inside the tolerance)
    differing = int(np.count_nonzero(np.any(sums != z["frame_checksums"], axis=1)))
    assert differing <= 1, f"{differing} frames differ from the fixture's"
    idx = z["delay_index"]
    np.testing.assert_array_equal(r["bin_counts"], z["bin_counts"])
    np.testing.assert_array_equal(r["pair_counts"][idx], z["pair_counts"])
    np.testing.assert_allclose(r["q_mean"], z["q_mean"], rtol=1e-12)
    ref, got = z["D"], r["D"][idx]
    m = (z["bin_counts"][None, :] > 0) & (z["pair_counts"][:, None] > 0)
    assert np.all(got[~m] == 0.0) and np.all(ref[~m] == 0.0)
    rel = np.abs(got[m] - ref[m]) / np.abs(ref[m])
    assert rel.max() <= TOL_F32, (float(rel.max()), np.unravel_index(np.argmax(np.where(m, np.abs(got - ref) / np.where(m, np.abs(ref), 1), 0)), m.shape))
    print(f"{name}: {int(m.sum())} binned values, max rel err {rel.max():.2e}, median {np.median(rel):.2e}")
