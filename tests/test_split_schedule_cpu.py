"""The accumulation schedule of the tensor-core GEMM (csrc/split_gemm.cu, make_schedule), read
through the host-only query bt_debug_split_schedule: no GPU work.

For S slices per operand the split product keeps the slice pairs (s, t) with s + t <= S + 1
(Ozaki et al., error-free splitting); over each K segment every such pair must be accumulated
exactly once, the pairs sharing one TMEM accumulator (lane) must have the same weight class
s + t, and each accumulator must stay an exact fp32 integer: a digit product is at most 2^12 in
magnitude, so n pairs over L blocks of 64 terms stay below n L 2^18, which must be below 2^24
(below 2^22, the magic-number conversion's range, for a lane drained that way)."""
import itertools

import pytest


@pytest.fixture(scope="module")
def pkg():
    from paper_2508_19138_gb300 import build
    build.build()
    import paper_2508_19138_gb300 as p
    return p


CASES = [(S, KB) for S in (2, 3, 4, 5, 6, 7, 8) for KB in (1, 2, 3, 5, 7, 8, 13, 15, 16, 31, 32, 45)]


def _segments(jobs):
    return sorted({(j[3], j[4]) for j in jobs})


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("S,KB", CASES)
def test_every_pair_once_per_segment_with_exact_lanes(pkg, mode, S, KB):
    r = pkg.bt_debug_split_schedule(S, KB, mode)
    assert r is not None
    jobs, items, F = r
    segs = _segments(jobs)
    # the segments tile [0, KB) and none is longer than 15 blocks
    assert segs[0][0] == 0 and segs[-1][1] == KB
    for (a0, a1), (b0, b1) in zip(segs, segs[1:]):
        assert a1 == b0
    assert all(0 < b - a <= 15 for a, b in segs)
    want = sorted((s, t) for s in range(1, S + 1) for t in range(1, S + 1) if s + t <= S + 1)
    seen = {seg: [] for seg in segs}
    for dual, ib, ie, kb0, kb1, cvt0, cvt1, _ in jobs:
        L = kb1 - kb0
        its = items[ib:ie]
        assert its, "empty job"
        lanes = [[(s, t) for s, _, t in its]]
        if dual:
            assert all(s2 == s + 1 for s, s2, _ in its)
            lanes.append([(s2, t) for _, s2, t in its])
        for lane, cvt in zip(lanes, (cvt0, cvt1)):
            assert len({s + t for s, t in lane}) == 1, lane  # one weight class per accumulator
            assert all(1 <= s <= S and 1 <= t <= S for s, t in lane)
            assert len(lane) * L < 64  # exact fp32 integer (below 2^24)
            if not cvt:
                assert len(lane) * L < 16  # inside the magic-number range (below 2^22)
            seen[(kb0, kb1)].extend(lane)
    for seg, pairs in seen.items():
        assert sorted(pairs) == want, (seg, sorted(pairs))
    assert F == min(7 * S - 9, 50 - (64 * KB - 1).bit_length())


def test_merged_schedule_drains_fewer_accumulators(pkg):
    """The merged schedule's drains per tile at the sweep's shapes (K' = 832 and 2048, 6 slices)."""
    def drains(S, KB, mode):
        jobs, _, _ = pkg.bt_debug_split_schedule(S, KB, mode)
        return len(jobs), sum(1 + j[0] for j in jobs)
    assert drains(6, 13, 1) == (12, 21)
    assert drains(6, 13, 0) == (7, 11)
    assert drains(6, 32, 1) == (36, 63)
    assert drains(6, 32, 0) == (18, 27)
    for S, KB in itertools.product(range(2, 9), (1, 3, 7, 8, 13, 32)):
        assert drains(S, KB, 0)[1] <= drains(S, KB, 1)[1]


def test_merged_jobs_longest_first(pkg):
    jobs, _, _ = pkg.bt_debug_split_schedule(6, 13, 0)
    cost = [(j[2] - j[1]) * (j[4] - j[3]) * (1 + j[0]) for j in jobs]
    assert cost == sorted(cost, reverse=True)


def test_unsupported_arguments(pkg):
    assert pkg.bt_debug_split_schedule(1, 13) is None
    assert pkg.bt_debug_split_schedule(9, 13) is None
    assert pkg.bt_debug_split_schedule(6, 0) is None
