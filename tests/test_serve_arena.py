"""The serving loop's budget arena (first fit, coalescing on release), host code only: a
randomised allocate / release sequence through a compiled driver against a plain Python
model of the same policy, with the invariants checked at every step (blocks inside the
budget and disjoint, free list sorted, disjoint and fully coalesced, in_use + free = size)."""
import os
import random
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2008_08483_gb300", "csrc")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("arena") / "arena_driver")
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, os.path.join(HERE, "arena_driver.cpp"),
                    "-o", exe], check=True)
    return exe


def model_alloc(free, size):
    """First fit over the sorted free list; returns the offset or None."""
    for i, (o, n) in enumerate(free):
        if n >= size:
            if n == size:
                free.pop(i)
            else:
                free[i] = (o + size, n - size)
            return o
    return None


def model_release(free, off, size):
    free.append((off, size))
    free.sort()
    out = []
    for o, n in free:
        if out and out[-1][0] + out[-1][1] == o:
            out[-1] = (out[-1][0], out[-1][1] + n)
        else:
            out.append((o, n))
    free[:] = out


def test_arena_matches_first_fit_model(driver):
    rng = random.Random(2024)
    size = 1 << 20
    ops, expect_allocs = ["init %d" % size], []
    free, live = [(0, size)], []
    in_use = peak = 0
    states = []
    for step in range(4000):
        if live and (rng.random() < 0.45 or len(live) > 40):
            off, n = live.pop(rng.randrange(len(live)))
            ops.append("free %d %d" % (off, n))
            model_release(free, off, n)
            in_use -= n
        else:
            n = 256 * rng.randint(1, 400)
            ops.append("alloc %d" % n)
            off = model_alloc(free, n)
            expect_allocs.append(-1 if off is None else off)
            if off is not None:
                live.append((off, n))
                in_use += n
                peak = max(peak, in_use)
        if step % 50 == 0:
            ops.append("state")
            states.append((in_use, peak, max([b for _, b in free], default=0), list(free)))
    out = subprocess.run([driver], input="\n".join(ops) + "\n", capture_output=True, text=True,
                         check=True).stdout.split("\n")
    got_allocs, got_states = [], []
    for line in out:
        if not line:
            continue
        parts = line.split()
        if len(parts) == 1:
            got_allocs.append(int(parts[0]))
        else:
            blocks = [tuple(int(v) for v in p.split(":")) for p in parts[3:]]
            got_states.append((int(parts[0]), int(parts[1]), int(parts[2]), blocks))
    assert got_allocs == expect_allocs
    assert got_states == states
    for iu, _, _, blocks in got_states:
        assert iu + sum(n for _, n in blocks) == size
        for (o1, n1), (o2, _) in zip(blocks, blocks[1:]):
            assert o1 + n1 < o2                      # sorted, disjoint, never adjacent
    assert any(a == -1 for a in got_allocs)          # the budget did run out at times


def test_arena_full_release_restores_one_block(driver):
    ops = ["init 4096", "alloc 1024", "alloc 1024", "alloc 2048", "alloc 1",
           "free 1024 1024", "free 0 1024", "free 2048 2048", "state"]
    out = subprocess.run([driver], input="\n".join(ops) + "\n", capture_output=True, text=True,
                         check=True).stdout.split()
    assert out[:4] == ["0", "1024", "2048", "-1"]
    assert out[4:] == ["0", "4096", "4096", "0:4096"]
