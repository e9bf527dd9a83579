"""The serving runtime's work-unit scheduler (csrc/unit_sched.h), compiled with g++ as host code:
round robin over requests at energy-chunk granularity, small units passing a unit that does not
fit, and the bound on how often the oldest waiting request can be passed."""
import os
import random
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2508_19138_gb300", "csrc")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("sched") / "sched_driver")
    subprocess.run([gxx, "-O1", "-std=c++17", "-I", CSRC, os.path.join(HERE, "sched_driver.cpp"), "-o", exe],
                   check=True, capture_output=True, text=True)
    return exe


def run(driver, entries, cmds, max_skips=4):
    lines = [f"E {len(entries)} {max_skips}"] + [" ".join(map(str, e)) for e in entries] + cmds
    r = subprocess.run([driver], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    return [int(x) for x in r.stdout.split()]


def test_round_robin_over_requests_at_chunk_granularity(driver):
    picks = run(driver, [(1, 3, 100), (2, 3, 100), (3, 3, 100)], ["P 1000"] * 10)
    assert picks == [0, 1, 2, 0, 1, 2, 0, 1, 2, -1]


def test_a_request_arriving_later_joins_the_rotation(driver):
    picks = run(driver, [(1, 4, 10), (2, 4, 10)], ["P 100", "P 100", "A 2 10", "P 100", "P 100", "P 100", "P 100"])
    assert picks == [0, 1, 0, 1, 2, 0]


def test_small_units_pass_one_that_does_not_fit(driver):
    picks = run(driver, [(1, 2, 500), (2, 2, 50), (3, 1, 60)], ["P 100", "P 100", "P 100", "P 1000", "P 1000"])
    assert picks == [1, 2, 1, 0, 0]


def test_the_head_is_passed_at_most_max_skips_times(driver):
    picks = run(driver, [(1, 1, 500), (2, 9, 10)], ["P 100"] * 5 + ["P 500", "P 100"], max_skips=3)
    assert picks == [1, 1, 1, -1, -1, 0, 1]


def model_pick(entries, max_skips, free):
    """The policy restated: the entry with the smallest order among those with units left (the
    head) if it fits; otherwise, unless it was passed max_skips times, the smallest-order other
    entry that fits (the head's pass count grows by one)."""
    live = [i for i, e in enumerate(entries) if e[1] > 0]
    if not live:
        return -1
    head = min(live, key=lambda i: entries[i][0])
    if entries[head][2] <= free:
        entries[head][3] = 0
        return head
    if entries[head][3] >= max_skips:
        return -1
    others = [i for i in live if i != head and entries[i][2] <= free]
    if not others:
        return -1
    entries[head][3] += 1
    return min(others, key=lambda i: entries[i][0])


@pytest.mark.parametrize("seed", range(6))
def test_random_sequences_against_the_restated_policy(driver, seed):
    rng = random.Random(seed)
    n = rng.randint(2, 7)
    entries = [[i + 1, rng.randint(1, 5), rng.choice([16, 64, 256, 1024])] for i in range(n)]
    frees = [rng.choice([32, 100, 300, 2000]) for _ in range(40)]
    got = run(driver, [tuple(e) for e in entries], [f"P {f}" for f in frees], max_skips=2)
    model = [e + [0] for e in entries]
    seq = 1000000
    want = []
    for f in frees:
        i = model_pick(model, 2, f)
        if i >= 0:
            model[i][1] -= 1
            seq += 1
            model[i][0] = seq
        want.append(i)
    assert got == want
