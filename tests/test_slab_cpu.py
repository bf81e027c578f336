"""Mode slabs on the host (no GPU): the slabs of a frame shape partition its 16-mode tiles in order,
and the shares of a binned average held by two gloo ranks add up, through the one all-reduce of
reduce_slabs, to the binning of the whole spectrum (Eq. 1 holds mode by mode, so the split is exact
up to the FP64 rounding of the sum)."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import paper_1209_3362_gb300 as P


@pytest.fixture(scope="module")
def lib():
    P.build()
    return P.load_library()


SHAPES = [(64, 64), (128, 96), (2048, 2048), (384, 512), (96, 768), (6, 4)]


@pytest.mark.parametrize("H,W", SHAPES)
def test_slabs_partition_the_tiles(lib, H, W):
    full = -(-H * (W // 2 + 1) // 16) * 16
    for n in (1, 2, 3, 7, 8):
        if n > full // 16:
            with pytest.raises(P.NFSError):
                P.slab_range(H, W, 0, n)
            continue
        ranges = [P.slab_range(H, W, s, n) for s in range(n)]
        assert ranges[0][0] == 0 and sum(m for _, m in ranges) == full
        for (a, m), (b, _) in zip(ranges, ranges[1:]):
            assert a + m == b
        assert all(a % 16 == 0 and m % 16 == 0 and m > 0 for a, m in ranges)
        sizes = [m for _, m in ranges]
        assert max(sizes) - min(sizes) <= 16  # tiles split evenly


def test_slab_range_rejects(lib):
    with pytest.raises(P.NFSError):
        P.slab_range(64, 64, 2, 2)
    with pytest.raises(P.NFSError):
        P.slab_range(64, 64, -1, 2)
    with pytest.raises(P.NFSError):
        P.slab_range(64, 64, 0, 0)
    with pytest.raises(P.NFSError):
        P.slab_range(64, 70, 0, 2)


def share(Dk, H, W, nq, first, n):
    """A slab's share of every bin average: sum over its modes of w_k D_k / C_b (host numpy)."""
    t = P.bin_table(H, W, nq)
    b, c = t["bin_of_mode"], t["bin_counts"]
    Wh = W // 2 + 1
    ky, kx = np.meshgrid(np.arange(H), np.arange(Wh), indexing="ij")
    k = kx * H + ky  # column-major mode order
    inside = (k >= first) & (k < first + n) & (b >= 0)
    w = np.where((kx == 0) | (kx == W // 2), 1.0, 2.0)
    out = np.zeros((Dk.shape[0], nq))
    for j in range(Dk.shape[0]):
        np.add.at(out[j], b[inside], (w * Dk[j])[inside])
    return out / np.where(c > 0, c, 1)[None, :], c


def _rank(rank, world, port, H, W, nq, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        Dk = np.random.default_rng(7).gamma(2.0, 1.0, size=(3, H, W // 2 + 1))  # the same on every rank
        first, n = P.slab_range(H, W, rank, world)
        part, c = share(Dk, H, W, nq, first, n)
        pc = np.array([10, 9, 5], np.int64)
        red = P.reduce_slabs({"D": part, "bin_counts": c, "pair_counts": pc}, group=dist.group.WORLD)
        whole, _ = share(Dk, H, W, nq, 0, 1 << 40)
        out[rank] = float(np.max(np.abs(red["D"] - whole) / np.maximum(np.abs(whole), 1e-300)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("H,W,nq", [(64, 96, 24), (128, 128, 64)])
def test_two_ranks_sum_their_slab_shares(lib, H, W, nq):
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, H, W, nq, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] <= 1e-13 and res[1] <= 1e-13


def test_reduce_slabs_in_one_process(lib):
    a = {"D": np.array([[1.0, 2.0]]), "bin_counts": np.array([3, 4]), "pair_counts": np.array([5])}
    b = {"D": np.array([[0.5, 0.25]]), "bin_counts": np.array([3, 4]), "pair_counts": np.array([5])}
    r = P.reduce_slabs([a, b])
    assert np.array_equal(r["D"], np.array([[1.5, 2.25]])) and np.array_equal(r["bin_counts"], a["bin_counts"])
