"""Tables of the thread-per-cell FP32 source-term kernel (host code only): chem_f32t_tables.h
through a compiled driver on the synthetic mechanisms, checked against the descriptor.
- Each record's centred Arrhenius form (Eq. 6 about 1000 K, head on the 2^-12 grid) gives
  log2 k(T).
- Each species record's centred Gibbs form (the powers of T re-expanded about its range's
  centre) gives -g/(RT) log2 e from NASA-7 (Eq. 10), in the right T range.
- The entries carry the stoichiometry as shared-row offsets, the falloff records the
  low-pressure limit and the Troe constants, and the quads' interleaved efficiency lists
  the listed efficiencies.
- The processing order holds every reaction once, grouped by type, padded to quads and to
  chunks of 16.
A mechanism with four species on a side is refused (the warp-per-cell kernel takes it)."""
import dataclasses
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2008_08483_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2008_08483_gb300", "csrc")
INC = os.path.join(os.path.dirname(HERE), "include")
LOG2E = 1.0 / math.log(2.0)
PF_ROW, OM_ROW = 384, 132                    # bytes per species row of the P/F and omega tables


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    cuda_inc = "/usr/local/cuda/include"
    if cxx is None or not os.path.isdir(cuda_inc):
        pytest.skip("no C++ compiler or CUDA headers")
    exe = str(tmp_path_factory.mktemp("f32t") / "f32t_tables_driver")
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, "-I", INC, "-I", cuda_inc,
                    os.path.join(HERE, "f32t_tables_driver.cpp"), "-o", exe], check=True)
    return exe


def run(exe, m):
    ns, nr = m.n_species, m.nu_f.shape[0]
    f = lambda a, fmt: " ".join(fmt % x for x in np.asarray(a).ravel())
    text = "\n".join([
        "%d %d %.17g %.17g" % (ns, nr, m.t_mid, m.p_ref), f(m.mol_weight, "%.17g"),
        f(m.nu_f, "%d"), f(m.nu_r, "%d"), f(m.arrh, "%.17g"), f(m.kind, "%d"),
        f(m.reversible, "%d"), f(m.eff, "%.17g"), f(m.arrh_low, "%.17g"), f(m.troe, "%.17g"),
        f(m.nasa7, "%.17g")]) + "\n"
    out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout
    lines = out.strip().splitlines()
    res = {"ok": int(lines[0].split()[1]), "rec": [], "spec": [], "tb": [], "fall": []}
    for ln in lines[1:]:
        tag, *vals = ln.split()
        if tag == "sizes":
            res["sizes"] = [int(x) for x in vals]
        elif tag == "const":
            res["const"] = np.array(vals, np.float32).astype(float)
        elif tag == "rec":
            res["rec"].append(vals)
        elif tag == "spec":
            res["spec"].append(np.array(vals, np.float32).astype(float))
        elif tag == "tb":
            res["tb"].append((int(vals[0]), float(np.float32(vals[1]))))
        elif tag == "fall":
            res["fall"].append(np.array(vals, np.float32).astype(float))
    return res


def parse_rec(v):
    j = int(v[0])
    kf = np.array(v[1:5], np.float32).astype(float)
    b = float(np.float32(v[5]))
    meta, tb = int(v[6]), int(v[7])
    rb = float(np.float32(v[8]))
    ent = [(int(v[9 + 2 * e]), float(np.float32(v[10 + 2 * e]))) for e in range(12)]
    return j, kf, b, meta, tb, rb, ent


def log2k_centred(kf, b, T):
    d1 = np.log2(T) - np.log2(1000.0)
    d2 = 1.0 / T - 1.0 / 1000.0
    return kf[0] + kf[1] + b * d1 + (kf[2] + kf[3]) * d2


def g_log2(a, T):
    """-g/(RT) log2 e from the NASA-7 set a (Eq. 10)."""
    return LOG2E * (a[0] * (np.log(T) - 1.0) + a[1] * T / 2 + a[2] * T**2 / 6 + a[3] * T**3 / 12
                    + a[4] * T**4 / 20 - a[5] / T + a[6])


@pytest.mark.parametrize("size", ["h2air_9_21", "gri_53_325", "heavy_160_1000"])
def test_tables_against_descriptor(driver, size):
    m = synth.make_mechanism(size, seed=1)
    ns, nr = m.n_species, m.nu_f.shape[0]
    res = run(driver, m)
    assert res["ok"] == 1
    n_rec, n_tb, n_fall, n_sp = res["sizes"]
    assert n_rec == len(res["rec"]) and n_rec % 16 == 0 and n_sp == ns
    # constants: (hi, lo) pairs of log2 1000, 1/1000, log2 R, log2(p_ref / R), log2 e
    R = 8.31446261815324e7
    c = res["const"]
    for (h, l), x in zip(c[:10].reshape(5, 2), [math.log2(1000.0), 1e-3, math.log2(R),
                                           math.log2(m.p_ref / R), LOG2E]):
        assert abs(h + l - x) <= 1e-12 * max(1.0, abs(x))
    recs = [parse_rec(v) for v in res["rec"]]
    seen = [j for j, *_ in recs if j >= 0]
    assert sorted(seen) == list(range(nr))
    Ts = np.array([300.0, 700.0, 999.0, 1000.0, 1500.0, 2600.0, 3500.0])
    nf_ = (m.nu_f > 0).sum(1)
    nr_ = (m.nu_r > 0).sum(1)
    types = []
    for i, (j, kf, b, meta, tb, rb, ent) in enumerate(recs):
        ty = meta & 7
        types.append(ty)
        if j < 0:
            assert kf[0] == -2000.0 and all(o == ns * PF_ROW or o == ns * OM_ROW for o, _ in ent)
            assert all(nu == 0.0 for _, nu in ent)
            continue
        kind = int(m.kind[j])
        want = (0 if nf_[j] <= 2 and nr_[j] <= 2 else 1) if kind == 0 else kind + 1
        assert ty == want
        # centred Arrhenius: head exact on the grid, and log2 k(T)
        assert kf[0] * 4096.0 == round(kf[0] * 4096.0) and abs(kf[0]) < 1024.0
        lnA, bb, EoR = m.arrh[j]
        ref = (lnA + bb * np.log(Ts) - EoR / Ts) * LOG2E
        assert np.max(np.abs(log2k_centred(kf, b, Ts) - ref)) <= 5e-7
        assert rb == (0.0 if m.reversible[j] else -2000.0)
        # entries: reactant slots 0, 1, 8; product slots 2, 3, 9; net slots 4-7, 10, 11
        react = [(k * PF_ROW, float(m.nu_f[j, k])) for k in range(ns) if m.nu_f[j, k]]
        prod = [(k * PF_ROW, float(m.nu_r[j, k])) for k in range(ns) if m.nu_r[j, k]]
        net = [(k * OM_ROW, float(m.nu_r[j, k] - m.nu_f[j, k])) for k in range(ns)
               if m.nu_r[j, k] != m.nu_f[j, k]]
        pad = lambda lst, n, z: lst + [(z, 0.0)] * (n - len(lst))
        assert [ent[p] for p in (0, 1, 8)] == pad(react, 3, ns * PF_ROW)
        assert [ent[p] for p in (2, 3, 9)] == pad(prod, 3, ns * PF_ROW)
        assert [ent[p] for p in (4, 5, 6, 7, 10, 11)] == pad(net, 6, ns * OM_ROW)
        if kind >= 2:
            f = res["fall"][meta >> 8]
            assert abs(f[0]) < 1024.0 and f[0] * 4096.0 == round(f[0] * 4096.0)
            lnA0, b0, E0 = m.arrh_low[j]
            ref0 = (lnA0 + b0 * np.log(Ts) - E0 / Ts) * LOG2E
            assert np.max(np.abs(log2k_centred(f[0:4], f[4], Ts) - ref0)) <= 5e-7
            if kind == 3:
                al, T3, T1, T2 = m.troe[j]
                Fc = (f[5] * 2.0 ** (Ts * f[7]) + f[6] * 2.0 ** (Ts * f[8])
                      + f[10] * 2.0 ** (f[9] / Ts))
                Fc_ref = ((1 - al) * np.exp(-Ts / T3) + al * np.exp(-Ts / T1)
                          + (np.exp(-T2 / Ts) if T2 > 0 else 0.0))
                assert np.max(np.abs(Fc / Fc_ref - 1.0)) <= 1e-5
    # grouped by type, in type order; quads of one type; padding only inside the last quad
    # of a type or after the last type (to the chunk)
    last = max(i for i, (j, *_ ) in enumerate(recs) if j >= 0)
    assert types[:last + 1] == sorted(types[:last + 1])
    for q in range(0, last + 1, 4):
        assert len(set(types[q:q + 4])) == 1
    # the quads' efficiency lists, interleaved [entry][reaction]
    for q in range(0, n_rec, 4):
        tbw = recs[q][4]
        base, nit = tbw & 0xFFFF, tbw >> 16
        for u in range(4):
            j = recs[q + u][0]
            lst = [(k * PF_ROW, float(np.float32(m.eff[j, k] - 1.0))) for k in range(ns)
                   if j >= 0 and m.kind[j] >= 1 and m.eff[j, k] != 1.0]
            got = [res["tb"][base + it * 4 + u] for it in range(nit)]
            assert got == lst + [(ns * PF_ROW, 0.0)] * (nit - len(lst))
        js = [recs[q + u][0] for u in range(4) if recs[q + u][0] >= 0]
        sets = [set(np.nonzero(m.nu_r[j] != m.nu_f[j])[0]) for j in js]
        disjoint = all(not (sets[a] & sets[b]) for a in range(len(sets))
                       for b in range(a + 1, len(sets)))
        if js:
            assert bool(recs[q][3] & 8) == disjoint
    # species: centred Gibbs form against NASA-7 in each T range, 1 / W
    for k in range(ns):
        s = res["spec"][k].reshape(2, 12)
        for rg, TT in ((0, Ts[Ts < m.t_mid]), (1, Ts[Ts >= m.t_mid])):
            ga, gb, gc = s[rg, 0:4], s[rg, 4:8], s[rg, 8:12]
            assert ga[0] * 4096.0 == round(ga[0] * 4096.0) and abs(ga[0]) < 1024.0
            d1 = np.log2(TT) - np.log2(1000.0)
            d2 = 1.0 / TT - 1e-3
            u = (TT - c[10 + rg]) / 1000.0        # the range's own centre
            G = (ga[0] + ga[1] + (ga[2] + ga[3]) * d1 + (gb[0] + gb[1]) * d2
                 + u * (gb[2] + u * (gb[3] + u * (gc[0] + u * gc[1]))))
            ref = g_log2(m.nasa7[k, rg], TT)
            # log2 units, absolute: the FP32 coefficients of the quartic in u leave
            # below 1e-6 (with a single centre at 1000 K: ~4e-6 at 3500 K)
            assert np.max(np.abs(G - ref)) <= 2e-6
            assert abs(gc[2] - 1.0 / m.mol_weight[k]) <= 1e-7 / m.mol_weight[k]


def test_four_reactants_refused(driver):
    base = synth.make_mechanism("gri_53_325", seed=1)
    j = int(np.nonzero((base.nu_f > 0).sum(1) == 3)[0][0])
    k = int(np.nonzero((base.nu_f[j] == 0) & (base.nu_r[j] == 0))[0][0])
    nu_f, nu_r = base.nu_f.copy(), base.nu_r.copy()
    nu_f[j, k] += 1
    nu_r[j, k] += 1
    m = dataclasses.replace(base, nu_f=nu_f, nu_r=nu_r)
    assert run(driver, m)["ok"] == 0
