"""The no-allocation entry point against the context entry points, through the C ABI.

nfs_structure_function_noalloc serves callers that cannot allocate device memory while they run
(device memory owned by another allocator, or acquisition loops that must not take the
synchronisation cudaMalloc / cudaFree can imply).  It takes its scratch from one static device
array that every call shares, so two calls in a row must each match what a fresh context gives
for the same frames: the second call must not see the first call's leftovers.  This file is named
to be collected last, so a failure here comes after every other test has run.
"""
import numpy as np
import pytest
import torch

import nfs_synth as S
import paper_1209_3362_gb300 as P

pytestmark = pytest.mark.gpu

TOL_F32 = 2e-5  # the tolerance of the fused FP32 path in the parity tests


def context_result(dev_frames, delays, nq):
    with P.NFS(dev_frames.shape[1], dev_frames.shape[2], delays, nq) as ctx:
        ctx.push_frames_device(dev_frames)
        return ctx.structure_function()


def compare(got, ref):
    np.testing.assert_array_equal(got["bin_counts"], ref["bin_counts"])
    np.testing.assert_array_equal(got["pair_counts"], ref["pair_counts"])
    R, D = ref["D"], got["D"]
    nz = R != 0
    assert np.all(D[~nz] == 0.0)
    assert np.max(np.abs(D[nz] - R[nz]) / np.abs(R[nz])) <= TOL_F32


def test_noalloc_matches_context_path_on_two_calls_in_a_row():
    assert torch.cuda.is_available()
    P.build()
    cases = [
        (S.OUFrameSource(128, 128, 0.5, seed=41).frames_numpy(80), list(range(1, 21)) + [40, 79], 64),
        (S.OUFrameSource(96, 64, 2.0, seed=42).frames_numpy(50), [1, 2, 3, 5, 8, 30, 60], 24),
        # 100 frames through a ring of R = 5 + 32 = 37 slots: the ring wraps, and 4-frame FFT chunks
        # straddle its last and first slots (37 is not a multiple of 4)
        (S.OUFrameSource(64, 64, 1.0, seed=43).frames_numpy(100), [1, 2, 3, 5], 16),
    ]
    for frames, delays, nq in cases:
        dev = torch.from_numpy(frames.view(np.int16)).cuda()
        ref = context_result(dev, delays, nq)
        got = P.structure_function_noalloc(dev, delays, nq)
        compare(got, ref)
    # the same first case again after the second: leftovers of the previous call must not leak
    frames, delays, nq = cases[0]
    dev = torch.from_numpy(frames.view(np.int16)).cuda()
    compare(P.structure_function_noalloc(dev, delays, nq), context_result(dev, delays, nq))


def test_noalloc_rejects_sizes_beyond_its_scratch():
    dev = torch.zeros((2, 1024, 1024), dtype=torch.int16, device="cuda")
    with pytest.raises(P.NFSError) as e:
        P.structure_function_noalloc(dev, [1, 100], 16)
    assert e.value.status == P.NFS_ETOOBIG


def test_noalloc_leaves_device_memory_unchanged():
    """After a first call (which loads the library's kernels and its static array), further calls
    change neither PyTorch's allocations nor the device's free memory."""
    fr = torch.from_numpy(S.OUFrameSource(64, 64, 1.0, seed=44).frames_numpy(40).view(np.int16)).cuda()
    P.structure_function_noalloc(fr, [1, 2, 7], 16)
    torch.cuda.synchronize()
    alloc0, free0 = torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]
    for _ in range(2):
        P.structure_function_noalloc(fr, [1, 2, 7], 16)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.cuda.mem_get_info()[0] == free0
