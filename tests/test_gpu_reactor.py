"""Constant-pressure reactor kernels (right-hand side, analytic Jacobian, Rosenbrock
integrator) through the C ABI against the oracle: its right-hand side and Jacobian, scipy
Radau integrations of its reactor, closed forms of toy mechanisms, and invariants.
Bars: 1e-10 per cell for the FP64 right-hand side and Jacobian; ignition delay within 0.1 %
of Radau (rtol 1e-10) at rtol 1e-6."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2008_08483_gb300 import build as B
from paper_2008_08483_gb300 import chem, synth

import reactor_toys as toys

pytestmark = pytest.mark.gpu
R = synth.R_CGS


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    B.build()
    return torch.device("cuda:0")


def t64(x, dev):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device=dev)


def _states(mech, n, seed):
    T, P, Y, _ = synth.make_ignition_states(mech, n, seed=seed)
    rng = np.random.default_rng(seed)
    Yb = 0.7 * Y + 0.3 * rng.dirichlet(np.full(mech.n_species, 0.3), n)
    Yb[:, rng.integers(0, mech.n_species, 5)] = 0.0
    Yb[0, 1] = -1e-12              # a slightly negative mass fraction, as an integrator makes
    return np.concatenate([T, T + 700]), np.concatenate([P, P]), np.concatenate([Y, Yb])


@pytest.mark.parametrize("size,n", [("h2air_9_21", 37), ("gri_53_325", 70),
                                    ("heavy_160_1000", 20)])
def test_rhs_and_jacobian_match_oracle(dev, size, n):
    m = synth.make_mechanism(size, seed=1)
    h = chem.Mechanism(m)
    om = O.OracleMechanism(m)
    T, P, Y = _states(m, n // 2, seed=7)
    f = chem.ode_rhs(h, t64(T, dev), t64(P, dev), t64(Y, dev)).cpu().numpy()
    J = chem.ode_jacobian(h, t64(T, dev), t64(P, dev), t64(Y, dev)).cpu().numpy()
    for i in range(len(T)):
        y = np.concatenate([[T[i]], Y[i]])
        fr = O.ode_rhs(om, P[i], y)
        assert abs(f[i, 0] - fr[0]) <= 1e-10 * abs(fr[0])
        assert np.max(np.abs(f[i, 1:] - fr[1:])) <= 1e-10 * np.max(np.abs(fr[1:]))
        Jr = O.ode_jac(om, P[i], y)
        for c in range(len(y)):
            sc = np.max(np.abs(Jr[:, c]))
            if sc > 0:
                assert np.max(np.abs(J[i, :, c] - Jr[:, c])) <= 1e-10 * sc, (i, c)


def test_jacobian_matches_central_differences_of_rhs(dev, mech53):
    h = chem.Mechanism(mech53)
    T, P, Y = _states(mech53, 2, seed=9)
    i = 2
    y = np.concatenate([[T[i]], Y[i]])
    n = len(y)
    steps = np.array([1e-4] + [1e-6 * max(abs(v), 1e-3) for v in y[1:]])
    yp = np.tile(y, (n, 1)) + np.diag(steps)
    ym = np.tile(y, (n, 1)) - np.diag(steps)
    Pv = np.full(n, P[i])
    fp = chem.ode_rhs(h, t64(yp[:, 0], dev), t64(Pv, dev), t64(yp[:, 1:], dev)).cpu().numpy()
    fm = chem.ode_rhs(h, t64(ym[:, 0], dev), t64(Pv, dev), t64(ym[:, 1:], dev)).cpu().numpy()
    Jfd = ((fp - fm) / (2 * steps[:, None])).T
    J = chem.ode_jacobian(h, t64(T[i:i + 1], dev), t64(P[i:i + 1], dev),
                          t64(Y[i:i + 1], dev)).cpu().numpy()[0]
    for c in range(n):
        sc = np.max(np.abs(Jfd[:, c]))
        assert np.max(np.abs(J[:, c] - Jfd[:, c])) <= 2e-5 * sc, c


def _integrate(h, T, P, Y, dev, t_end, **kw):
    Tt, Pt, Yt = t64(T, dev), t64(P, dev), t64(Y, dev)
    out = chem.integrate(h, Tt, Pt, Yt, t_end, **kw)
    torch.cuda.synchronize()
    res = {k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in out.items()}
    res["T"], res["Y"] = Tt.cpu().numpy(), Yt.cpu().numpy()
    return res


def test_convergence_order_on_linear_problem(dev):
    # A <=> B is a linear ODE; with fixed steps the global error falls as h^3 (order 3)
    k, da7 = 1.0, 1.0
    h = chem.Mechanism(toys.isomerisation(k, da7))
    errs = []
    for H in (0.1, 0.05, 0.025):
        r = _integrate(h, [1200.0], [2e6], [[0.9, 0.1]], dev, 1.0, rtol=1e3, atol=1e3,
                       h_init=H, h_max=H)
        assert r["status"][0] == 0 and r["n_rejected"][0] == 0
        assert r["n_accepted"][0] == round(1.0 / H)
        errs.append(abs(r["Y"][0, 0] - toys.isomerisation_exact(k, da7, 0.9, 1.0)))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all((orders > 2.8) & (orders < 3.2)), orders


def test_fp32_stage_jacobian(dev, mech53, ignition53):
    """The FP32 stage Jacobian (opt-in) against the FP64 one on 256 reactors of the
    autoignition batch integrated to 1 ms at rtol 1e-6: both are error-controlled to the
    same tolerance, so ignition delays agree within 0.1 %, end states within 5e-5 (each run
    is within 1e-5 of Radau at rtol 1e-10 on the reference reactors), and step counts within
    10 %."""
    h = chem.Mechanism(mech53)
    T, P, Y = (a[::16] for a in ignition53)
    a = _integrate(h, T, P, Y, dev, 1e-3, rtol=1e-6, atol=1e-12, jacobian_fp32=True)
    b = _integrate(h, T, P, Y, dev, 1e-3, rtol=1e-6, atol=1e-12)
    assert np.all(a["status"] == 0) and np.all(b["status"] == 0)
    ig = b["t_ign"] > 0
    assert np.array_equal(a["t_ign"] > 0, ig)
    assert np.max(np.abs(a["t_ign"][ig] / b["t_ign"][ig] - 1.0)) < 1e-3
    assert np.max(np.abs(a["T"] / b["T"] - 1.0)) < 5e-5
    assert np.max(np.abs(a["Y"] - b["Y"])) < 5e-5
    assert abs(a["n_accepted"].sum() / b["n_accepted"].sum() - 1.0) < 0.1
    h.close()


def test_fixed_steps_mode(dev, mech53):
    # fixed_steps = K takes K equal steps without error control: the same arithmetic as an
    # adaptive run pinned to h = t_end / K with a tolerance every step passes
    k, da7 = 1.0, 1.0
    h = chem.Mechanism(toys.isomerisation(k, da7))
    a = _integrate(h, [1200.0], [2e6], [[0.9, 0.1]], dev, 1.0, fixed_steps=10)
    b = _integrate(h, [1200.0], [2e6], [[0.9, 0.1]], dev, 1.0, rtol=1e3, atol=1e3,
                   h_init=0.1, h_max=0.1)
    assert a["n_accepted"][0] == 10 and a["n_rejected"][0] == 0 and a["status"][0] == 0
    assert np.array_equal(a["Y"], b["Y"]) and np.array_equal(a["T"], b["T"])
    # one step of 1e-8 s across the violent initial transients of detonation-channel states
    # (no error control: the result need not be accurate): a cell either gets a finite state
    # or CHEM_CELL_NONFINITE with its input state kept
    hm = chem.Mechanism(mech53)
    T, P, Y = synth.make_znd_states(mech53, 256, seed=4)
    r = _integrate(hm, T, P, Y, dev, 1e-8, fixed_steps=1)
    ok = r["status"] == chem.CELL_OK
    assert np.all(ok | (r["status"] == chem.CELL_NONFINITE)) and ok.any()
    assert np.all(np.isfinite(r["Y"][ok])) and np.all(np.isfinite(r["T"][ok]))
    assert np.array_equal(r["Y"][~ok], Y[~ok]) and np.array_equal(r["T"][~ok], T[~ok])
    assert r["failed"] == (not ok.all())


def test_dimerisation_closed_form(dev):
    k, T, P = 1e12, 1500.0, 3e6
    h = chem.Mechanism(toys.dimerisation(k))
    for t_end in (1e-7, 1e-6, 1e-5):
        r = _integrate(h, [T], [P], [[1.0, 0.0]], dev, t_end, rtol=1e-9, atol=1e-15)
        exact = toys.dimerisation_exact(k, T, P, [t_end])[0]
        assert abs(r["Y"][0, 0] - exact) / exact < 1e-6
        assert abs(r["T"][0] - T) < 1e-8


def test_exothermic_invariant_and_ignition(dev):
    dh = 20000.0
    m = toys.exothermic(lnA=14.0, EoR=10000.0, dh=dh)
    h = chem.Mechanism(m)
    r = _integrate(h, [1000.0], [1e6], [[1.0, 0.0]], dev, 2e-3, rtol=1e-6, atol=1e-12)
    assert abs(r["T"][0] - (1000.0 + dh / 3.5 * (1.0 - r["Y"][0, 0]))) < 1e-6
    ref = O.integrate_reactor(O.OracleMechanism(m), 1000.0, 1e6, [1.0, 0.0], 2e-3)
    assert abs(r["t_ign"][0] / ref["t_ign"] - 1.0) < 1e-3


@pytest.fixture(scope="module")
def ignition53(dev, mech53):
    T, P, Y, _ = synth.make_ignition_states(mech53, 4096, seed=1234)
    return T, P, Y


def test_ignition_delay_matches_radau(dev, mech53, ignition53):
    T, P, Y = ignition53
    sel = [0, 1, 2, 3]
    h = chem.Mechanism(mech53)
    r = _integrate(h, T[sel], P[sel], Y[sel], dev, 1e-2, rtol=1e-6, atol=1e-12)
    assert np.all(r["status"] == 0)
    om = O.OracleMechanism(mech53)
    for q, i in enumerate(sel):
        ref = O.integrate_reactor(om, T[i], P[i], Y[i], 1e-2, rtol=1e-10, atol=1e-20)
        assert np.isfinite(ref["t_ign"]) and r["t_ign"][q] > 0
        assert abs(r["t_ign"][q] / ref["t_ign"] - 1.0) < 1e-3, (i, r["t_ign"][q], ref["t_ign"])
        assert abs(r["T"][q] / ref["y_end"][0] - 1.0) < 1e-5
        assert np.max(np.abs(r["Y"][q] - ref["y_end"][1:])) < 1e-5


@pytest.mark.parametrize("j32", [False, True], ids=["jacobian_fp64", "jacobian_fp32"])
def test_ignition_delay_over_the_batch(dev, mech53, ignition53, j32):
    """A fixed sample of the 4096-reactor autoignition batch (T0 strata, the extremes of T0,
    P0 and phi, and reactors that do not ignite by 10 ms), integrated to 10 ms at rtol 1e-6:
    the ignition delay within 0.1 % of the oracle's Radau run (rtol 1e-10), a reactor that
    does not ignite there not reported as ignited, and every reactor's 10 ms state within
    1e-5 (tests/golden/ignition_53_325.json, from make_ignition_reference.py)."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "ignition_53_325.json")) as f:
        ref = json.load(f)
    assert ref["mechanism"] == {"size": "gri_53_325", "seed": 1}
    assert ref["states"]["n"] == len(ignition53[0])
    idx = np.array(ref["index"])
    T, P, Y = (a[idx] for a in ignition53)
    assert len(idx) >= 32 and sum(t is None for t in ref["t_ign"]) >= 2
    h = chem.Mechanism(mech53)
    r = _integrate(h, T, P, Y, dev, ref["t_end"], rtol=1e-6, atol=1e-12, jacobian_fp32=j32)
    assert np.all(r["status"] == 0)
    for q, (t_ref, y_ref) in enumerate(zip(ref["t_ign"], ref["y_end"])):
        if t_ref is None:
            assert not r["t_ign"][q] > 0, (idx[q], r["t_ign"][q])
        else:
            assert abs(r["t_ign"][q] / t_ref - 1.0) < 1e-3, (idx[q], r["t_ign"][q], t_ref)
        assert abs(r["T"][q] / y_ref[0] - 1.0) < 1e-5, (idx[q], r["T"][q], y_ref[0])
        assert np.max(np.abs(r["Y"][q] - np.asarray(y_ref[1:]))) < 1e-5, idx[q]
    h.close()


def test_invariants_along_the_batch(dev, mech53, ignition53):
    T, P, Y = ignition53
    n = 512
    h = chem.Mechanism(mech53)
    r = _integrate(h, T[:n], P[:n], Y[:n], dev, 1e-3, rtol=1e-6, atol=1e-12)
    assert np.all(r["status"] == 0)
    assert np.max(np.abs(r["Y"].sum(1) - 1.0)) < 1e-9
    el0 = (Y[:n] / mech53.mol_weight) @ mech53.elem_comp
    el1 = (r["Y"] / mech53.mol_weight) @ mech53.elem_comp
    assert np.max(np.abs(el1 - el0)) / np.max(np.abs(el0)) < 1e-9
    om = O.OracleMechanism(mech53)
    for i in range(0, n, 64):
        _, h0, _, _ = O.thermo(om, T[i])
        _, h1, _, _ = O.thermo(om, r["T"][i])
        H0 = np.sum(Y[i] * R * T[i] * h0 / mech53.mol_weight)
        H1 = np.sum(r["Y"][i] * R * r["T"][i] * h1 / mech53.mol_weight)
        cp_scale = R * 5.0 * r["T"][i] / np.min(mech53.mol_weight)
        assert abs(H1 - H0) < 1e-4 * cp_scale
    assert np.all(r["T"] > T[:n])      # every reactor ignited and burnt


def test_result_independent_of_batch(dev, mech53, ignition53):
    T, P, Y = ignition53
    h = chem.Mechanism(mech53)
    full = _integrate(h, T[:96], P[:96], Y[:96], dev, 1e-4)
    for i in (0, 37, 95):
        one = _integrate(h, T[i:i + 1], P[i:i + 1], Y[i:i + 1], dev, 1e-4)
        assert one["T"][0] == full["T"][i] and np.array_equal(one["Y"][0], full["Y"][i])
        assert one["n_accepted"][0] == full["n_accepted"][i]


def test_failed_cells_report_status(dev, mech53, ignition53):
    T, P, Y = ignition53
    h = chem.Mechanism(mech53)
    r = _integrate(h, T[:8], P[:8], Y[:8], dev, 1e-2, max_steps=3)
    assert r["failed"] and np.all(r["status"] == chem.CELL_MAX_STEPS)
    with pytest.raises(chem.ChemError) as e:
        _integrate(h, T[:8], P[:8], Y[:8], dev, 1e-2, max_steps=3, raise_on_failure=True)
    assert e.value.status == 8
    # t_end = 0 leaves the state unchanged
    r = _integrate(h, T[:8], P[:8], Y[:8], dev, 0.0)
    assert not r["failed"] and np.array_equal(r["T"], T[:8]) and np.array_equal(r["Y"], Y[:8])
    assert np.all(r["t_ign"] == -1.0)


def test_large_mechanism_uses_global_matrices(dev, mech160):
    T, P, Y, _ = synth.make_ignition_states(mech160, 3, seed=5)
    h = chem.Mechanism(mech160)
    r = _integrate(h, T, P, Y, dev, 2e-8, rtol=1e-6, atol=1e-12)
    assert np.all(r["status"] == 0)
    om = O.OracleMechanism(mech160)
    for i in range(3):
        ref = O.integrate_reactor(om, T[i], P[i], Y[i], 2e-8, rtol=1e-10, atol=1e-20)
        assert abs(r["T"][i] / ref["y_end"][0] - 1.0) < 1e-5
        assert np.max(np.abs(r["Y"][i] - ref["y_end"][1:])) < 1e-5


def test_argument_errors(dev, mech9):
    h = chem.Mechanism(mech9)
    L = chem.lib()
    T = t64([1500.0], dev)
    P = t64([1e6], dev)
    Y = t64(np.full((1, 9), 1.0 / 9), dev)
    st = chem.CELL_OK
    for args in [(-1, 9, 1e-3, 1e-6, 1e-12), (1, 8, 1e-3, 1e-6, 1e-12), (1, 9, -1.0, 1e-6, 1e-12),
                 (1, 9, 1e-3, 0.0, 1e-12), (1, 9, 1e-3, 1e-6, -1.0)]:
        n, ld, te, rt, at = args
        rc = L.chem_integrate_cells(h.handle, n, T.data_ptr(), P.data_ptr(), Y.data_ptr(), ld,
                                    te, rt, at, None, None, None)
        assert rc == 1, args
    assert L.chem_ode_rhs(h.handle, 1, T.data_ptr(), P.data_ptr(), Y.data_ptr(), 9, None, 10,
                          None) == 1
    assert L.chem_ode_rhs(h.handle, 1, T.data_ptr(), P.data_ptr(), Y.data_ptr(), 9,
                          Y.data_ptr(), 9, None) == 1
    assert st == 0
