"""Safety of the fused delay kernel's copy schedule, checked on the host for many delay lists (no
GPU): the kernel streams older frames through a ring of shared-memory rows (frame f in row f mod
rows) in copy groups that a producer issues ahead of the computing warps.  For every step the rows
must hold exactly the frames the step reads, and no group may be issued (need) while an
unfinished step still reads a row it overwrites; a group's barrier may be re-armed only after the
group that last used it was consumed.  Also covers the shifted passes of the out-of-core mode,
where the block's frames and the older frames belong to different sequences."""
import numpy as np
import pytest

import nfs_synth as S
import paper_1209_3362_gb300 as P


@pytest.fixture(scope="module", autouse=True)
def _lib():
    P.build()
    P.load_library()


def _simulate(delays, cross, sc=None):
    sc = sc or P.delay_schedule(delays, cross)
    K, SB, F = sc["block_frames"], sc["slot_rows"], sc["copy_barriers"]
    sr, st = sc["subruns"], sc["stages"]
    # every delay appears once, in order, in runs of consecutive values of at most 16
    flat = [d0 + i for (_, ln, d0) in sr for i in range(ln)]
    assert flat == [d for d in delays if cross or d != 0]
    assert all(1 <= ln <= 16 for (_, ln, _) in sr)
    G = len(st) + 1
    glo = [0] + [int(s[2]) for s in st]
    ghi = [K - 1] + [int(s[3]) for s in st]
    need = [0] + [int(s[4]) for s in st]
    nlo, nhi = [0], [K - 1]  # frames each step reads (relative to t0)
    for s in st:
        first, n = int(s[0]), int(s[1])
        dmin, dmax = int(sr[first][2]), int(sr[first + n - 1][2] + sr[first + n - 1][1] - 1)
        assert K + dmax - dmin <= SB
        nlo.append(-dmax)
        nhi.append(K - 1 - dmin)
    seq = lambda step: 1 if (cross and step == 0) else 0  # noqa: E731  (block vs older sequence)
    for g in range(G):
        assert need[g] <= g  # a group never waits for the step that needs it
        if g >= F:
            assert need[g] >= g - F + 1  # its barrier's previous group was consumed
        if glo[g] > ghi[g]:
            continue
        f = np.arange(glo[g], ghi[g] + 1)
        for q in range(need[g], g):  # steps that may still run when group g is issued
            h = np.arange(nlo[q], nhi[q] + 1)
            rows_h = {int(r): int(x) for r, x in zip(np.mod(h, SB), h)}
            for r, x in zip(np.mod(f, SB), f):
                y = rows_h.get(int(r))
                if y is not None:
                    assert y == x and seq(g) == seq(q), (cross, g, q, int(x), y)
    # replay the groups in order: each step finds its frames (identity = sequence and index)
    ring = {}
    for q in range(G):
        for x in range(glo[q], ghi[q] + 1):
            ring[x % SB] = (seq(q), x)
        for y in range(nlo[q], nhi[q] + 1):
            assert ring.get(y % SB) == (seq(q), y), (cross, q, y)
    return len(st)


LISTS = [
    S.log_delays(1, 2000, 200), S.log_delays(1, 500, 100), S.log_delays(1, 250, 64), S.log_delays(1, 1200, 70),
    list(range(1, 51)), list(range(1, 600)), [0, 1, 2, 5, 11, 30], [1000, 1010], [1, 2, 3, 400, 401, 900, 1250],
    [300, 301, 302, 700, 5000, 5001, 9000], [5], list(range(7, 4200, 7)), list(range(184, 445, 3)),
]


@pytest.mark.parametrize("cross", [False, True])
@pytest.mark.parametrize("i", range(len(LISTS)))
def test_schedule_is_safe(cross, i):
    assert _simulate(LISTS[i], cross) >= 1


def _random_lists(n, seed):
    """Seeded delay lists of mixed structure: dense runs, sparse delays with random gaps, clusters
    of short runs far apart, and log spacing with random ends."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n):
        kind = i % 4
        if kind == 0:  # runs of random length separated by random gaps
            d, x = [], int(rng.integers(1, 40))
            while len(d) < int(rng.integers(5, 250)):
                d.extend(range(x, x + int(rng.integers(1, 30))))
                x = d[-1] + 1 + int(rng.integers(1, 200))
        elif kind == 1:  # isolated delays with random gaps (some shorter than a run of 16)
            d = list(np.cumsum(rng.integers(1, 120, size=int(rng.integers(2, 150)))))
        elif kind == 2:  # a few clusters far apart
            d = sorted({int(c) + j for c in rng.integers(1, 8000, size=6) for j in range(int(rng.integers(1, 20)))})
        else:  # log spacing with random ends and counts
            hi = int(rng.integers(50, 4000))
            d = S.log_delays(1, hi, int(rng.integers(10, min(hi, 220))))
        out.append([int(v) for v in d if 1 <= v <= 60000])
    return out


@pytest.mark.parametrize("cross", [False, True])
def test_random_delay_lists_are_safe(cross):
    """120 seeded delay lists of mixed structure; lists too long for the kernel's schedule (which
    then runs the one-thread-per-mode kernel) are refused by the export and skipped."""
    checked = 0
    for d in _random_lists(120, 20260 + int(cross)):
        try:
            sc = P.delay_schedule(d, cross)
        except P.NFSError:
            continue
        assert _simulate(d, cross, sc) >= 1
        checked += 1
    assert checked >= 90


def test_cross_schedule_with_delay_zero():
    # a shifted pass pairs frame u with the other sequence's frame u: delay 0 is computed
    sc = P.delay_schedule([0, 300, 301, 700], cross=True)
    assert sc["subruns"][0][2] == 0
    _simulate([0, 300, 301, 700], True)


def test_check_catches_an_early_group():
    """The check is not vacuous: issuing one group a step earlier than the schedule allows (a row
    still being read gets overwritten) is caught."""
    d = S.log_delays(1, 2000, 200)
    sc = P.delay_schedule(d)
    st = sc["stages"]
    g = next(i for i in range(len(st)) if st[i][4] > max(0, (i + 1) - sc["copy_barriers"] + 1))
    bad = dict(sc, stages=st.copy())
    bad["stages"][g][4] -= 1
    with pytest.raises(AssertionError):
        _simulate(d, False, bad)


@pytest.mark.parametrize("span", [16, 64, 112, 176, 320, 400, 512])
@pytest.mark.parametrize("cross", [False, True])
def test_every_stage_span_is_safe(span, cross):
    """The stage span the autotuner may choose regroups sub-runs into copy stages; every span keeps
    the replay's invariants on named and seeded lists, and the sub-runs (hence the pair arithmetic
    and the partial-sum batches) do not depend on it."""
    lists = [S.log_delays(1, 2000, 200), list(range(1, 129)), list(range(64, 2049, 64)), S.log_delays(1, 500, 100)]
    lists += _random_lists(20, 4242 + span + int(cross))
    checked = 0
    for d in lists:
        try:
            sc = P.delay_schedule(d, cross, span=span)
            ref = P.delay_schedule(d, cross)
        except P.NFSError:
            continue
        assert np.array_equal(sc["subruns"], ref["subruns"])
        for s in sc["stages"]:  # no stage spans more than `span` delays
            first, n = int(s[0]), int(s[1])
            lo = int(sc["subruns"][first][2])
            hi = int(sc["subruns"][first + n - 1][2] + sc["subruns"][first + n - 1][1] - 1)
            assert hi - lo <= max(span, int(sc["subruns"][first][1]) - 1)
        assert _simulate(d, cross, sc) >= 1
        checked += 1
    assert checked >= 15


def test_span_limits():
    with pytest.raises(P.NFSError):
        P.delay_schedule([1, 2, 3], span=15)
    with pytest.raises(P.NFSError):
        P.delay_schedule([1, 2, 3], span=513)
