"""Reference ignition delays and 10 ms end states of a fixed sample of the 53/325 autoignition
batch (ignition_53_325.json), from the CPU oracle's reactor integrated with scipy Radau.

The batch is the 4096 constant-pressure reactors of the autoignition workload
(synth.make_ignition_states, mechanism gri_53_325 seed 1, states seed 1234: T0 ~ U[900, 1400]
K, P0 ~ U[1, 20] atm, phi ~ U[0.5, 2]), integrated to t = 10 ms.  The sample is chosen from the
inputs alone:
  - 24 reactors spread over T0 (the middle reactor of each of 24 equal T0 bins),
  - the reactors with the smallest and largest T0, P0 and phi,
  - the coolest, lowest-pressure reactors (smallest sum of T0 and P0 ranks), added until at
    least two of the sample do not ignite by 10 ms.
Ignition delay: the first time T reaches T0 + 400 K (the integrator's reading of the paper's
ignition, located on Radau's dense output); reactors that do not ignite are compared on
their state at 10 ms.

Calls only the oracle (and the input generator).  Run it to rewrite the fixture:
  python tests/golden/make_ignition_reference.py
"""
import json
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

SIZE, MECH_SEED, STATE_SEED, N, T_END = "gri_53_325", 1, 1234, 4096, 1e-2
RTOL, ATOL = 1e-10, 1e-20
OUT = os.path.join(HERE, "ignition_53_325.json")


def states():
    from paper_2008_08483_gb300 import synth
    m = synth.make_mechanism(SIZE, seed=MECH_SEED)
    T, P, Y, phi = synth.make_ignition_states(m, N, seed=STATE_SEED)
    return m, T, P, Y, phi


def spread_sample(T, P, phi):
    """Input-only choice: T0 strata, then the extremes of T0, P0 and phi (in that order)."""
    order = np.argsort(T, kind="stable")
    bins = np.array_split(order, 24)
    idx = [int(b[len(b) // 2]) for b in bins]
    for a in (T, P, phi):
        for j in (int(np.argmin(a)), int(np.argmax(a))):
            if j not in idx:
                idx.append(j)
    return idx


def cool_candidates(T, P):
    """Reactors by increasing sum of T0 and P0 ranks (the likeliest not to ignite)."""
    rank = np.argsort(np.argsort(T)) + np.argsort(np.argsort(P))
    return [int(i) for i in np.argsort(rank, kind="stable")]


def _one(i):
    from oracle import oracle as O
    m, T, P, Y, _ = states()
    r = O.integrate_reactor(O.OracleMechanism(m), T[i], P[i], Y[i], T_END, rtol=RTOL, atol=ATOL)
    return i, r["t_ign"], r["y_end"].tolist(), r["nsteps"]


def main():
    _, T, P, _, phi = states()
    idx = spread_sample(T, P, phi)
    ctx = mp.get_context("spawn")
    res = {}
    with ctx.Pool(min(len(idx), os.cpu_count() or 4)) as pool:
        for i, t_ign, y, ns in pool.imap_unordered(_one, idx):
            res[i] = (t_ign, y, ns)
            print(f"reactor {i}: t_ign {t_ign:.6e} s, {ns} steps", flush=True)
        cand = [i for i in cool_candidates(T, P) if i not in res]
        while sum(1 for v in res.values() if not np.isfinite(v[0])) < 2 and cand:
            batch, cand = cand[:8], cand[8:]
            for i, t_ign, y, ns in pool.imap_unordered(_one, batch):
                res[i] = (t_ign, y, ns)
                print(f"reactor {i}: t_ign {t_ign:.6e} s, {ns} steps", flush=True)
    keys = sorted(res)
    doc = {
        "about": "oracle reactor (scipy Radau, rtol 1e-10, atol 1e-20) on a fixed sample of the "
                 "53/325 autoignition batch; written by make_ignition_reference.py",
        "mechanism": {"size": SIZE, "seed": MECH_SEED},
        "states": {"n": N, "seed": STATE_SEED},
        "t_end": T_END, "ign_dT": 400.0, "rtol": RTOL, "atol": ATOL,
        "index": keys,
        "t_ign": [res[i][0] if np.isfinite(res[i][0]) else None for i in keys],
        "y_end": [res[i][1] for i in keys],
        "steps": [res[i][2] for i in keys],
    }
    with open(OUT, "w") as f:
        json.dump(doc, f, indent=0)
    n_no = sum(1 for i in keys if not np.isfinite(res[i][0]))
    print(f"wrote {OUT}: {len(keys)} reactors, {n_no} without ignition by {T_END} s")


if __name__ == "__main__":
    main()
