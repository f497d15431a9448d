"""Order of the reactions for the thread-per-cell FP32 kernel (host code only): the quad plan
of chem_quads.h through a compiled driver, against a plain Python model of the same rule,
with its invariants checked on random mechanisms and on the synthetic ones.

Rule: per type, greedy packing in reaction order into the first open quad whose net species
are disjoint from its members'; full quads first (flagged disjoint), then the rest in order,
four to a quad (flagged disjoint only if they are), the last one padded with -1."""
import os
import random
import shutil
import subprocess

import numpy as np
import pytest

from paper_2008_08483_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2008_08483_gb300", "csrc")
NTYPES = 5


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("quads") / "quads_driver")
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, os.path.join(HERE, "quads_driver.cpp"),
                    "-o", exe], check=True)
    return exe


def run_driver(exe, types, nets):
    lines = ["%d %d" % (NTYPES, len(types))]
    lines += ["%d %d %s" % (t, len(n), " ".join(map(str, n))) for t, n in zip(types, nets)]
    out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True,
                         check=True).stdout
    return [tuple(int(x) for x in ln.split()) for ln in out.strip().splitlines() if ln.strip()]


def model(types, nets):
    plan = []
    for g in range(NTYPES):
        open_q = []
        for j, t in enumerate(types):
            if t != g:
                continue
            for q in open_q:
                if len(q[0]) < 4 and not (q[1] & set(nets[j])):
                    q[0].append(j)
                    q[1].update(nets[j])
                    break
            else:
                open_q.append([[j], set(nets[j])])
        rest = []
        for members, _ in open_q:
            if len(members) == 4:
                plan.append((g, 1, *members))
            else:
                rest += members
        for a in range(0, len(rest), 4):
            chunk = rest[a:a + 4]
            seen, dis = set(), True
            for j in chunk:
                dis = dis and not (seen & set(nets[j]))
                seen |= set(nets[j])
            plan.append((g, int(dis), *(chunk + [-1] * (4 - len(chunk)))))
    return plan


def check_invariants(plan, types, nets):
    slots = [s for q in plan for s in q[2:]]
    real = [s for s in slots if s >= 0]
    assert sorted(real) == list(range(len(types)))            # every reaction exactly once
    assert [q[0] for q in plan] == sorted(q[0] for q in plan)  # grouped, in type order
    for i, (g, dis, *members) in enumerate(plan):
        live = [j for j in members if j >= 0]
        assert live and all(types[j] == g for j in live)
        assert members == live + [-1] * (4 - len(live))        # padding at the end only
        if len(live) < 4:                                      # ... of the type's last quad
            assert i + 1 == len(plan) or plan[i + 1][0] != g
        sets = [set(nets[j]) for j in live]
        pairwise = all(not (sets[a] & sets[b]) for a in range(len(sets))
                       for b in range(a + 1, len(sets)))
        assert bool(dis) == pairwise


def test_random_mechanisms(driver):
    rng = random.Random(7)
    for case in range(60):
        ns = rng.randint(2, 64)
        nr = rng.randint(1, 180)
        types = [rng.choice([0, 0, 0, 1, 2, 4]) if case % 3 else rng.randrange(NTYPES)
                 for _ in range(nr)]
        nets = [sorted(rng.sample(range(ns), rng.randint(1, min(6, ns)))) for _ in range(nr)]
        got = run_driver(driver, types, nets)
        assert got == model(types, nets)
        check_invariants(got, types, nets)


@pytest.mark.parametrize("size", ["h2air_9_21", "gri_53_325"])
def test_synthetic_mechanisms(driver, size):
    """The kernel's grouping of the synthetic mechanisms (elementary with at most two species
    a side, other elementary, third-body, Lindemann, Troe): nearly every quad of 53/325 is
    disjoint; 9 species leave few disjoint quads but lose no reaction."""
    m = synth.make_mechanism(size, seed=1)
    nf = (m.nu_f > 0).sum(1)
    nr = (m.nu_r > 0).sum(1)
    types = [int(0 if (k == 0 and a <= 2 and b <= 2) else 1 if k == 0 else k + 1)
             for k, a, b in zip(m.kind, nf, nr)]
    nets = [list(np.nonzero(m.nu_r[j] != m.nu_f[j])[0]) for j in range(len(types))]
    got = run_driver(driver, types, nets)
    assert got == model(types, nets)
    check_invariants(got, types, nets)
    if size == "gri_53_325":
        assert sum(q[1] for q in got) >= 0.9 * len(got)
