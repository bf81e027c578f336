"""The benchmark's algorithmic counts (the numerators of its roofline figures), checked on the
host: pairs per pass against the closed sum, and bytes per launch against a brute-force count of
the ring slots and accumulators a block touches."""
import bench
import nfs_synth as S


def test_pairs_equal_the_closed_sum():
    w = S.WORKLOADS["ddm2048"]
    _, launches, pairs = bench.delay_block_bytes(w.delays, w.N, 512, 1)
    assert pairs == sum(max(0, w.N - d) for d in w.delays) == 741785
    assert launches == 8


def test_block_bytes_brute_force():
    N, K, M = 11, 4, 3
    delays = [0, 1, 3, 9]
    total, launches, pairs = bench.delay_block_bytes(delays, N, K, M)
    want, want_pairs = 0, 0
    for t0 in range(0, N, K):
        block = range(t0, min(N, t0 + K))
        active = [d for d in delays if d <= block[-1]]
        slots = set(block)
        for d in active:
            for t in block:
                if t - d >= 0:
                    slots.add(t - d)
                    want_pairs += 1
        want += 8 * M * len(slots) + 16 * M * len(active)
    assert (total, launches, pairs) == (want, 3, want_pairs)
    assert pairs == sum(max(0, N - d) for d in delays)
