"""Serving loop through the C ABI: results identical alone and in a concurrent mix (cells are
independent), identical to the direct entry points, FP64 source term within 1e-10 of the
oracle, admission by the HBM budget (refusal only above the whole budget, waiting for memory
otherwise), integration step counts, poll time-outs, continuous batching with graph replay and
in-place graph updates, and shutdown with abandoned tickets."""
import threading

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2008_08483_gb300 import build as B
from paper_2008_08483_gb300 import chem, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    B.build()
    m9 = synth.make_mechanism("h2air_9_21", seed=1)
    m53 = synth.make_mechanism("gri_53_325", seed=1)
    h9, h53 = chem.Mechanism(m9), chem.Mechanism(m53)
    srv = chem.Server([h9, h53], 2 << 30)
    yield dict(mechs=[m9, m53], handles=[h9, h53], srv=srv)
    srv.close()


def make_requests(mechs, n_req, seed, max_cells=3000):
    rng = np.random.default_rng(seed)
    reqs = []
    for q in range(n_req):
        mi = int(rng.integers(0, 2))
        m = mechs[mi]
        n = int(np.exp(rng.uniform(np.log(64), np.log(max_cells))))
        T, P, Y = synth.make_znd_states(m, n, seed=seed * 1000 + q)
        kind = chem.REQ_INTEGRATE if rng.uniform() < 0.4 else chem.REQ_SOURCE
        prec = chem.FP64 if kind == chem.REQ_INTEGRATE else \
            [chem.FP64, chem.FP32, chem.SPLIT_BF16][int(rng.integers(0, 3))]
        dt = np.float64 if prec == chem.FP64 else np.float32
        fixed = 0
        reqs.append(dict(mi=mi, kind=kind, prec=prec, fixed=fixed, T=T.astype(dt),
                         P=P.astype(dt), Y=np.ascontiguousarray(Y.astype(dt))))
    return reqs


def _submit(srv, r):
    T, P, Y = r["T"].copy(), r["P"].copy(), r["Y"].copy()
    if r["kind"] == chem.REQ_SOURCE:
        out = np.zeros_like(Y)
        t = srv.submit(r["mi"], r["kind"], T, P, Y, r["prec"], out=out)
        return t, dict(omega=out)
    st = np.full(T.shape[0], -1, np.int32)
    t = srv.submit(r["mi"], r["kind"], T, P, Y, chem.FP64, dt=1e-8, rtol=1e-6, atol=1e-12,
                   status=st, fixed_steps=r.get("fixed", 0))
    return t, dict(T=T, Y=Y, status=st)


def run_alone(srv, reqs):
    outs = []
    for r in reqs:
        t, o = _submit(srv, r)
        res = srv.poll(t, -1)
        assert res["status"] == 0, res
        outs.append(o)
    return outs


def run_mixed(srv, reqs, n_threads=8):
    outs = [None] * len(reqs)
    res = [None] * len(reqs)

    def rank(k):
        mine = list(range(k, len(reqs), n_threads))
        tick = {}
        for i in mine:
            tick[i], outs[i] = _submit(srv, reqs[i])
        for i in mine:
            res[i] = srv.poll(tick[i], -1)

    th = [threading.Thread(target=rank, args=(k,)) for k in range(n_threads)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=600)
    assert all(r is not None and r["status"] == 0 for r in res), res
    return outs, res


def test_alone_equals_mix(env):
    srv = env["srv"]
    reqs = make_requests(env["mechs"], 40, seed=3)
    alone = run_alone(srv, reqs)
    mixed, res = run_mixed(srv, reqs)
    for a, b in zip(alone, mixed):
        for k in a:
            assert np.array_equal(a[k], b[k]), k
    assert max(r["batch_requests"] for r in res) >= 1


def test_served_equals_direct_calls(env):
    srv, hs = env["srv"], env["handles"]
    reqs = make_requests(env["mechs"], 12, seed=5)
    outs = run_alone(srv, reqs)
    dev = torch.device("cuda:0")
    for r, o in zip(reqs, outs):
        h = hs[r["mi"]]
        T, P, Y = (torch.as_tensor(a, device=dev) for a in (r["T"], r["P"], r["Y"]))
        if r["kind"] == chem.REQ_SOURCE:
            w = chem.source_term(h, T, P, Y, r["prec"]).cpu().numpy()
            assert np.array_equal(w, o["omega"])
        else:
            chem.integrate(h, T, P, Y, 1e-8, rtol=1e-6, atol=1e-12, fixed_steps=r["fixed"])
            assert np.array_equal(T.cpu().numpy(), o["T"])
            assert np.array_equal(Y.cpu().numpy(), o["Y"])
            assert np.all(o["status"] == 0)


def test_served_fp64_source_matches_oracle(env):
    srv, m = env["srv"], env["mechs"][1]
    T, P, Y = synth.make_znd_states(m, 700, seed=17)
    out = np.zeros_like(Y)
    t = srv.submit(1, chem.REQ_SOURCE, T, P, Y, chem.FP64, out=out)
    assert srv.poll(t, -1)["status"] == 0
    ref = O.source_term(m, T, P, Y)
    err = np.abs(out - ref).max(1) / np.abs(ref).max(1)
    assert err.max() <= 1e-10


def test_admission_and_errors(env):
    srv, m = env["srv"], env["mechs"][0]
    # a request needing more than the whole budget is refused at once: 16 MiB hold
    # 104857 cells of the 9-species FP64 source term ((2 + 2 * 9) * 8 bytes per cell)
    small = chem.Server([env["handles"][0]], 16 << 20)
    try:
        n = (16 << 20) // 160 + 1
        T, P = np.full(n, 1000.0), np.full(n, 1e6)
        Y = np.zeros((n, m.n_species))
        out = np.zeros_like(Y)
        with pytest.raises(chem.ChemError) as e:
            small.submit(0, chem.REQ_SOURCE, T, P, Y, chem.FP64, out=out)
        assert e.value.status == 2                     # over budget: CHEM_ENOMEM
    finally:
        small.close()
    T, P, Y = synth.make_znd_states(m, 8, seed=1)
    out = np.zeros_like(Y)
    with pytest.raises(chem.ChemError) as e:
        srv.submit(5, chem.REQ_SOURCE, T[:8], P[:8], Y[:8], chem.FP64, out=out[:8])
    assert e.value.status == 1
    with pytest.raises(chem.ChemError) as e:
        srv.submit(0, chem.REQ_INTEGRATE, T[:8].astype(np.float32), P[:8].astype(np.float32),
                   Y[:8].astype(np.float32), chem.FP32, dt=1e-8)
    assert e.value.status == 1
    with pytest.raises(chem.ChemError) as e:
        srv.poll(987654321, 0)
    assert e.value.status == 1


def test_poll_timeout_then_completion(env):
    srv, m = env["srv"], env["mechs"][1]
    T, P, Y, _ = synth.make_ignition_states(m, 2048, seed=3)
    st = np.zeros(2048, np.int32)
    t = srv.submit(1, chem.REQ_INTEGRATE, T, P, Y, chem.FP64, dt=2e-6, status=st)
    with pytest.raises(chem.ChemError) as e:
        srv.poll(t, 0)
    assert e.value.status == 7                         # CHEM_ENOTREADY
    with pytest.raises(chem.ChemError) as e:
        srv.poll(t, 1)
    assert e.value.status == 6                         # CHEM_ETIMEOUT
    res = srv.poll(t, -1)
    assert res["status"] == 0 and res["n_cells"] == 2048 and res["latency_us"] > 0
    with pytest.raises(chem.ChemError) as e:
        srv.poll(t, 0)                                 # released
    assert e.value.status == 1


def test_continuous_batching_and_graph_replay(env):
    srv = env["srv"]
    before = srv.info()
    reqs = [r for r in make_requests(env["mechs"], 64, seed=11, max_cells=200)]
    for r in reqs:
        r.update(kind=chem.REQ_SOURCE, mi=1, prec=chem.FP32)
        m = env["mechs"][1]
        T, P, Y = synth.make_znd_states(m, r["T"].shape[0], seed=int(r["T"].shape[0]))
        r.update(T=T.astype(np.float32), P=P.astype(np.float32),
                 Y=np.ascontiguousarray(Y.astype(np.float32)))
    tick = [_submit(srv, r) for r in reqs]
    res = [srv.poll(t, -1) for t, _ in tick]
    after = srv.info()
    assert all(r["status"] == 0 for r in res)
    assert after["max_batch_requests"] > 1            # requests queued meanwhile share a batch
    assert after["batches"] - before["batches"] < len(reqs)
    assert after["graph_launches"] - before["graph_launches"] == after["batches"] - before["batches"]
    assert after["graphs_captured"] >= 1
    assert after["graph_updates"] > before["graph_updates"]   # same key: graph updated in place


def test_admission_waits_for_memory(env):
    """Two requests that do not fit in the budget together: the second waits until the first
    retires (no refusal, no split into fixed slots), and both results equal the direct call."""
    h53, m = env["handles"][1], env["mechs"][1]
    n = 20000                                          # 20000 * (2 + 2 * 53) * 8 B = 17.3 MB
    srv = chem.Server([h53], 24 << 20)
    try:
        states = [synth.make_znd_states(m, n, seed=40 + q) for q in range(2)]
        outs = [np.zeros_like(Y) for _, _, Y in states]
        # submitted back to back, so the second arrives while the first holds its memory
        tick = [srv.submit(0, chem.REQ_SOURCE, T, P, Y, chem.FP64, out=o)
                for (T, P, Y), o in zip(states, outs)]
        reqs = [(T, P, Y, o, t) for (T, P, Y), o, t in zip(states, outs, tick)]
        res = [srv.poll(t, -1) for *_, t in reqs]
        info = srv.info()
        assert all(r["status"] == 0 and r["batch_requests"] == 1 for r in res)
        assert info["memory_waits"] >= 1
        assert info["bytes_in_use"] == 0 and 0 < info["bytes_in_use_max"] <= 24 << 20
        dev = torch.device("cuda:0")
        for T, P, Y, out, _ in reqs:
            w = chem.source_term(h53, *(torch.as_tensor(a, device=dev) for a in (T, P, Y)), chem.FP64)
            assert np.array_equal(w.cpu().numpy(), out)
    finally:
        srv.close()


def test_source_term_not_held_behind_integration(env):
    """A source-term request submitted while a long integration runs completes first: the
    source-term lanes have SMs of their own."""
    srv, m = env["srv"], env["mechs"][1]
    info = srv.info()
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    assert info["source_sms"] >= 8 and info["integrate_sms"] >= 8
    assert info["source_sms"] + info["integrate_sms"] <= nsm
    T, P, Y, _ = synth.make_ignition_states(m, 4096, seed=9)
    st = np.zeros(4096, np.int32)
    ti = srv.submit(1, chem.REQ_INTEGRATE, T, P, Y, chem.FP64, dt=5e-6, status=st)
    Ts, Ps, Ys = synth.make_znd_states(m, 1000, seed=8)
    Ts, Ps, Ys = Ts.astype(np.float32), Ps.astype(np.float32), np.ascontiguousarray(Ys.astype(np.float32))
    out = np.zeros_like(Ys)
    ts = srv.submit(1, chem.REQ_SOURCE, Ts, Ps, Ys, chem.SPLIT_BF16, out=out)
    rs = srv.poll(ts, -1)
    with pytest.raises(chem.ChemError) as e:
        srv.poll(ti, 0)
    assert e.value.status == 7                         # the integration is still running
    ri = srv.poll(ti, -1)
    assert rs["status"] == 0 and ri["status"] == 0
    assert rs["latency_us"] < ri["latency_us"]
    dev = torch.device("cuda:0")
    h53 = env["handles"][1]
    w = chem.source_term(h53, *(torch.as_tensor(a, device=dev) for a in (Ts, Ps, Ys)), chem.SPLIT_BF16)
    assert np.array_equal(w.cpu().numpy(), out)


def test_integration_step_counts(env):
    srv, m = env["srv"], env["mechs"][1]
    T, P, Y = synth.make_znd_states(m, 300, seed=23)
    st = np.full(300, -1, np.int32)
    t = srv.submit(1, chem.REQ_INTEGRATE, T, P, Y, chem.FP64, dt=1e-8, rtol=1e-6, atol=1e-12,
                   status=st)
    res = srv.poll(t, -1)
    assert res["status"] == 0 and np.all(st == 0)
    assert res["steps_accepted"] >= 300 and res["steps_rejected"] >= 0


def test_shutdown_with_abandoned_tickets(env):
    h9 = env["handles"][0]
    srv = chem.Server([h9], 256 << 20)
    T, P, Y = synth.make_znd_states(env["mechs"][0], 500, seed=2)
    outs = []
    for _ in range(10):
        o = np.zeros_like(Y)
        srv.submit(0, chem.REQ_SOURCE, T, P, Y, chem.FP64, out=o)
        outs.append(o)
    done = threading.Event()

    def close():
        srv.close()
        done.set()

    th = threading.Thread(target=close)
    th.start()
    assert done.wait(60), "destroy did not return"
