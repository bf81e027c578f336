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


def test_oracle_sample_takes_the_jobs_own_delay_prefix():
    """The timed oracle samples (reference arm and cpu_baseline leg) use the job's first n frames
    and the job's own delays below n, with at most the target number of pairs."""
    w = S.WORKLOADS["ddm2048"]
    n, delays, pairs = bench.sample_shape(w.delays, 100, 64)
    assert delays == [d for d in w.delays if d < n] and pairs == sum(n - d for d in delays) <= 100
    n2, _, pairs2 = bench.sample_shape(w.delays, 101 + pairs, 64)
    assert n2 > n and pairs2 > pairs
    n3, d3, _ = bench.sample_shape(S.WORKLOADS["paper512"].delays, 10 ** 9, 40)
    assert n3 == 40 and d3 == list(range(1, 40))


def test_reference_arm_prints_its_line():
    import json
    import subprocess
    import sys
    out = subprocess.run([sys.executable, bench.__file__, "--impl", "reference", "--workload", "ddm128", "--steps", "2",
                          "--warmup", "1", "--ref-budget", "0.3"], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["config"]["workload"] == "ddm128"


def test_binned_modes_equal_the_oracle_bin_table():
    """The roofline's flops count the binned modes only: the count equals the oracle's bin table
    (modes with a bin), and a slab's counts add up to the whole frame's."""
    import numpy as np
    import oracle
    import paper_1209_3362_gb300 as P
    oracle.build()
    P.load_library()
    for H, W, nq in [(64, 96, 24), (128, 128, 64), (96, 64, 40)]:
        bin_of, _, _ = oracle.bins(H, W, nq)
        want = int(np.count_nonzero(np.asarray(bin_of) >= 0))
        assert bench.binned_modes(P, H, W, nq) == want
        M = H * (W // 2 + 1)
        parts = [bench.binned_modes(P, H, W, nq, first, n) for first, n in
                 (P.slab_range(H, W, s, 3) for s in range(3))]
        assert sum(parts) == want and 0.7 * M < want < 0.85 * M
