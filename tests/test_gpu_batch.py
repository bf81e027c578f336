"""Ragged batch: sequences of uneven frame shapes and delay lists analysed together (one persistent
delay-update launch per block for all of them) must give, per sequence, what a single context
gives (bit for bit: the same arithmetic in the same order) and match the FP64 oracle."""
import numpy as np
import pytest
import torch

import nfs_synth as S
import paper_1209_3362_gb300 as P

pytestmark = pytest.mark.gpu

TOL_F32 = 2e-5


def rel_err(got, ref):
    m = (ref["bin_counts"][None, :] > 0) & (ref["pair_counts"][:, None] > 0) & (ref["D"] != 0)
    assert np.all(got["D"][~m & (ref["D"] == 0)] == 0.0)
    return float(np.max(np.abs(got["D"][m] - ref["D"][m]) / np.abs(ref["D"][m])))


@pytest.fixture(scope="module")
def ragged(oracle_lib):
    P.build()
    shapes = [(64, 64), (96, 128), (128, 128), (48, 64), (64, 96), (128, 96)]
    Ns = [300, 280, 530, 290, 310, 270]
    delays = [S.log_delays(1, 250, 30), list(range(1, 40)), S.log_delays(1, 250, 64), [1, 2, 3, 50, 120],
              S.log_delays(1, 200, 20) + [260], list(range(2, 30, 3))]
    nqs = [min(h, w) // 2 for h, w in shapes]
    frames = [S.OUFrameSource(h, w, 0.5 + 0.7 * i, seed=300 + i).frames_numpy(n)
              for i, ((h, w), n) in enumerate(zip(shapes, Ns))]
    refs = [oracle_lib.structure_function(f, d, q) for f, d, q in zip(frames, delays, nqs)]
    return shapes, delays, nqs, frames, refs


def test_batch_host_pushes_match_oracle_and_single_contexts(ragged):
    shapes, delays, nqs, frames, refs = ragged
    with P.NFSBatch(shapes, delays, nqs) as b:
        offs = [0] * len(shapes)  # round-robin pushes in uneven chunks
        chunk = [37, 64, 100, 13, 256, 80]
        while any(o < f.shape[0] for o, f in zip(offs, frames)):
            for s, f in enumerate(frames):
                if offs[s] < f.shape[0]:
                    n = min(chunk[s], f.shape[0] - offs[s])
                    b.push_frames(s, f[offs[s]:offs[s] + n])
                    offs[s] += n
        got = [b.structure_function(s) for s in range(len(shapes))]
    for s in range(len(shapes)):
        np.testing.assert_array_equal(got[s]["bin_counts"], refs[s]["bin_counts"])
        np.testing.assert_array_equal(got[s]["pair_counts"], refs[s]["pair_counts"])
        assert rel_err(got[s], refs[s]) <= TOL_F32, s
        with P.NFS(shapes[s][0], shapes[s][1], delays[s], nqs[s]) as ctx:
            ctx.push_frames(frames[s])
            single = ctx.structure_function()
        np.testing.assert_array_equal(got[s]["D"], single["D"])


def test_batch_device_push_all_at_once(ragged):
    shapes, delays, nqs, frames, refs = ragged
    dev = [torch.from_numpy(f.view(np.int16)).cuda() for f in frames]
    with P.NFSBatch(shapes, delays, nqs) as b:
        for s in range(len(shapes)):
            assert 1 <= b.member_option(s, P.OPT_FFT_CHUNK) <= 32  # chosen by the autotuner
        b.push_frames_device(dev)
        got = [b.structure_function(s) for s in range(len(shapes))]
        b.reset()
        b.push_frames_device([d[:100] for d in dev])
        got2 = [b.structure_function(s) for s in range(len(shapes))]
    for s in range(len(shapes)):
        assert rel_err(got[s], refs[s]) <= TOL_F32, s
        assert got2[s]["pair_counts"].max() <= 99


@pytest.fixture(scope="module")
def camera_shapes(oracle_lib):
    """The ragged workload's six camera shapes (128^2 .. 1024^2, radix-3 ones included), 520 frames
    each so that every member completes a 512-frame block and the persistent batched delay kernel
    runs over the large members' tiles, 12 log delays 1..260 and n_q = min(H, W) / 2."""
    P.build()
    shapes = [(1024, 1024), (768, 1024), (384, 512), (512, 512), (256, 256), (128, 128)]
    delays = [S.log_delays(1, 260, 12)] * len(shapes)
    nqs = [min(h, w) // 2 for h, w in shapes]
    frames = [S.OUFrameSource(h, w, 0.3 + 0.9 * i, seed=700 + i).frames_numpy(520) for i, (h, w) in enumerate(shapes)]
    refs = [oracle_lib.structure_function(f, d, q) for f, d, q in zip(frames, delays, nqs)]
    return shapes, delays, nqs, frames, refs


def test_batch_of_camera_shapes_matches_oracle(camera_shapes):
    shapes, delays, nqs, frames, refs = camera_shapes
    dev = [torch.from_numpy(f.view(np.int16)).cuda() for f in frames]
    with P.NFSBatch(shapes, delays, nqs) as b:
        b.push_frames_device(dev)
        got = [b.structure_function(s) for s in range(len(shapes))]
    for s in range(len(shapes)):
        np.testing.assert_array_equal(got[s]["bin_counts"], refs[s]["bin_counts"])
        np.testing.assert_array_equal(got[s]["pair_counts"], refs[s]["pair_counts"])
        assert rel_err(got[s], refs[s]) <= TOL_F32, (shapes[s], rel_err(got[s], refs[s]))
        with P.NFS(shapes[s][0], shapes[s][1], delays[s], nqs[s]) as ctx:
            ctx.push_frames_device(dev[s])
            single = ctx.structure_function()
        np.testing.assert_array_equal(got[s]["D"], single["D"])


def test_ragged48_workload_matches_oracle_on_its_small_members(oracle_lib):
    """The ragged benchmark workload itself (48 sequences x 500 frames of the six camera shapes, 64
    log delays 1..250 and min(H, W)/2 bins each, frames generated on the GPU as the benchmark does)
    in one batch: every member's bin and pair counts equal the oracle's, and the members of 128^2
    and 256^2 frames match the FP64 oracle's D within 2e-5."""
    P.build()
    rw = S.RAGGED_WORKLOADS["ragged48"]
    mem = rw.members()
    frames = []
    for (H, W, Dc, d, nq, seed) in mem:
        src = S.OUFrameSource(H, W, Dc, seed=seed, device="cuda", dtype=torch.float32)
        f = torch.empty((rw.N, H, W), dtype=torch.int16, device="cuda")
        for o in range(0, rw.N, 50):
            f[o:o + 50] = src.next_frames(min(50, rw.N - o))
        frames.append(f)
    torch.cuda.synchronize()
    with P.NFSBatch([(m[0], m[1]) for m in mem], [m[3] for m in mem], [m[4] for m in mem]) as b:
        b.push_frames_device(frames)
        got = [b.structure_function(s) for s in range(len(mem))]
    small = [s for s, m in enumerate(mem) if m[0] * m[1] <= 256 * 256]
    assert len(small) >= 8
    for s, (H, W, Dc, d, nq, seed) in enumerate(mem):
        table = P.bin_table(H, W, nq)
        np.testing.assert_array_equal(got[s]["bin_counts"], table["bin_counts"])
        np.testing.assert_array_equal(got[s]["pair_counts"], [max(0, rw.N - t) for t in d])
    for s in small:
        H, W, Dc, d, nq, seed = mem[s]
        ref = oracle_lib.structure_function(frames[s].cpu().numpy().view(np.uint16), d, nq)
        np.testing.assert_array_equal(got[s]["bin_counts"], ref["bin_counts"])
        assert rel_err(got[s], ref) <= TOL_F32, (s, H, W, rel_err(got[s], ref))
