"""The serving arena (first-fit device-memory arena of the request loop, csrc/arena.h), compiled
with g++ as host code and driven by random alloc/release sequences.  With a coalescing free list
the free space is exactly the gaps between live blocks, so first-fit must return the lowest-offset
gap of at least the request rounded up to 256 bytes: the model below computes that from the live
blocks alone and the arena must agree on every offset, never overlap, never exceed its size, and
give the whole arena back once everything is released."""
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
    exe = str(tmp_path_factory.mktemp("arena") / "arena_driver")
    subprocess.run([gxx, "-O1", "-std=c++17", "-I", CSRC, os.path.join(HERE, "arena_driver.cpp"), "-o", exe],
                   check=True, capture_output=True, text=True)
    return exe


def run(driver, lines):
    r = subprocess.run([driver], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    return [int(x) for x in r.stdout.split()]


def first_fit(live, size, capacity):
    """Lowest offset of a gap between live blocks (offset -> rounded length) that holds size."""
    need = (size + 255) // 256 * 256
    pos = 0
    for off in sorted(live):
        if off - pos >= need:
            return pos
        pos = max(pos, off + live[off])
    return pos if capacity - pos >= need else -1


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_arena_matches_first_fit_model(driver, seed):
    rng = random.Random(seed)
    capacity = rng.choice([1 << 20, 3 * (1 << 20) + 512, 10_000_000])
    # one scripted session: arena_driver's answers are compared afterwards, so the script must not
    # depend on them -- the model decides which blocks are live
    cmds = [f"reset {capacity}"]
    expected = []
    live = {}
    for _ in range(600):
        if live and rng.random() < 0.45:
            off = rng.choice(sorted(live))
            cmds.append(f"release {off} {live.pop(off)}")
        else:
            size = rng.choice([1, 255, 256, 257, 4096, rng.randint(1, capacity // 6), rng.randint(1, capacity // 40)])
            off = first_fit(live, size, capacity)
            cmds.append(f"alloc {size}")
            expected.append(off)
            if off >= 0:
                live[off] = (size + 255) // 256 * 256
    for off in sorted(live):
        cmds.append(f"release {off} {live.pop(off)}")
    cmds.append(f"alloc {capacity}")
    expected.append(0)
    got = run(driver, cmds)
    assert got == expected


def test_arena_no_overlap_and_alignment(driver):
    rng = random.Random(9)
    capacity = 1 << 22
    cmds = [f"reset {capacity}"] + [f"alloc {rng.randint(1, 50_000)}" for _ in range(200)]
    got = run(driver, cmds)
    blocks = []
    for line, off in zip(cmds[1:], got):
        size = int(line.split()[1])
        if off < 0:
            continue
        assert off % 256 == 0
        blocks.append((off, off + (size + 255) // 256 * 256))
    blocks.sort()
    assert blocks[-1][1] <= capacity
    assert all(a[1] <= b[0] for a, b in zip(blocks, blocks[1:]))
    # contiguous from 0 while nothing is released
    assert blocks[0][0] == 0 and all(a[1] == b[0] for a, b in zip(blocks, blocks[1:]))


def test_arena_coalesces_neighbours(driver):
    """Releasing the middle block, then its neighbours, leaves one free range that fits the sum."""
    cmds = ["reset 3072", "alloc 1024", "alloc 1024", "alloc 1024", "release 1024 1024", "alloc 2048",
            "release 0 1024", "alloc 2048", "release 2048 1024", "release 0 2048", "alloc 3072"]
    assert run(driver, cmds) == [0, 1024, 2048, -1, 0, 0]
