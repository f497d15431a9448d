"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a hand-worked
example (tests/golden), closed forms, thermodynamic identities, conservation
laws, detailed balance, limits of the falloff forms, and the paper's matrix form
(tests/matrix_form.py).
"""
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2008_08483_gb300 import synth

from matrix_form import source_term_tc as matrix_source_term_tc

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300))


def toy_mechanism(kind1=synth.KIND_THIRD_BODY, troe1=(0.0, 0.0, 0.0, 0.0), low1=(0.0, 0.0, 0.0)):
    """The worked example of tests/golden/toy_3sp_2rx.json as a Mechanism."""
    nasa = np.zeros((3, 2, 7))
    for k, (a1, a6, a7) in enumerate([(2.5, 30000.0, 5.0), (3.5, 0.0, 4.0), (4.5, 10000.0, 3.0)]):
        for r in range(2):
            nasa[k, r, 0], nasa[k, r, 5], nasa[k, r, 6] = a1, a6, a7
    eff = np.ones((2, 3))
    eff[0] = (1.0, 2.0, 1.0)
    arrh_low = np.zeros((2, 3))
    arrh_low[0] = low1
    troe = np.zeros((2, 4))
    troe[0] = troe1
    return synth.Mechanism(
        name="toy", elements=["X"], species=["X", "X2", "X3"],
        elem_comp=np.array([[1], [2], [3]], np.int32), mol_weight=np.array([10.0, 20.0, 30.0]),
        nu_f=np.array([[2, 0, 0], [1, 1, 0]], np.int32),
        nu_r=np.array([[0, 1, 0], [0, 0, 1]], np.int32),
        arrh=np.array([[np.log(1e15), -1.0, 0.0], [np.log(1e12), 0.5, 5000.0]]),
        kind=np.array([kind1, 0], np.int32), reversible=np.array([1, 1], np.int32),
        eff=eff, arrh_low=arrh_low, troe=troe, nasa7=nasa, t_mid=1000.0, p_ref=1e6)


@pytest.fixture(scope="module")
def golden_toy():
    with open(os.path.join(GOLDEN, "toy_3sp_2rx.json")) as f:
        g = json.load(f)
    ex = {k: (np.array([float(x) for x in v]) if isinstance(v, list) else float(v))
          for k, v in g["expected"].items()}
    return g, ex


# ---------------------------------------------------------------------------
# worked example
# ---------------------------------------------------------------------------

def test_toy_worked_example(golden_toy):
    g, ex = golden_toy
    m = toy_mechanism()
    st = g["state"]
    C = O.concentrations(m, st["T"], st["P"], ex["Y"])
    assert _rel(C, ex["C"]) < 1e-14
    assert _rel(O.thermo(m, st["T"])[3], ex["g_RT"]) < 1e-14
    d = O.cell_detail(m, st["T"], C)
    assert _rel(d["lnkf"], ex["lnkf"]) < 1e-14
    assert _rel(d["lnKc"], ex["lnKc"]) < 1e-14
    assert abs(d["M"][0] / ex["M"] - 1) < 1e-14
    assert _rel(d["qf"], ex["qf"]) < 1e-13
    assert _rel(d["qr"], ex["qr"]) < 1e-13
    assert _rel(d["omega"], ex["omega"]) < 1e-13
    w = O.source_term(m, [st["T"]], [st["P"]], ex["Y"][None, :])
    assert _rel(w[0], ex["omega"]) < 1e-13
    assert abs(np.dot(w[0], m.mol_weight)) < 1e-12 * np.dot(np.abs(w[0]), m.mol_weight)


def test_toy_troe_with_unit_fcent_is_lindemann(golden_toy):
    """alpha = 1, T* -> infinity, T** absent gives F_cent = 1, hence F = 1 (Lindemann)."""
    g, ex = golden_toy
    st = g["state"]
    low = (np.log(1e18), -1.5, 100.0)
    ml = toy_mechanism(synth.KIND_LINDEMANN, low1=low)
    mt = toy_mechanism(synth.KIND_TROE, troe1=(1.0, 100.0, 1e300, 0.0), low1=low)
    C = O.concentrations(ml, st["T"], st["P"], ex["Y"])
    dl, dt = O.cell_detail(ml, st["T"], C), O.cell_detail(mt, st["T"], C)
    assert _rel(dt["kf"], dl["kf"]) < 1e-15
    # Lindemann by hand: k = k_inf Pr/(1+Pr), Pr = k0 M / k_inf
    T = st["T"]
    kinf = 1e15 / T
    k0 = 1e18 * T ** -1.5 * np.exp(-100.0 / T)
    Pr = k0 * ex["M"] / kinf
    assert abs(dl["kf"][0] / (kinf * Pr / (1 + Pr)) - 1) < 1e-13


# ---------------------------------------------------------------------------
# closed forms and limits
# ---------------------------------------------------------------------------

def test_arrhenius_closed_forms():
    m = toy_mechanism(kind1=0)
    m.arrh[0] = (np.log(3.7e13), 0.0, 0.0)            # b = 0, E = 0: k = A at any T
    m.arrh[1] = (np.log(2.0e11), 1.5, 4000.0)
    C = np.array([1e-6, 2e-6, 3e-6])
    for T in (500.0, 1234.5, 3000.0):
        d = O.cell_detail(m, T, C)
        assert abs(d["kf"][0] / 3.7e13 - 1) < 1e-14
        # k(2T)/k(T) = 2^b exp(E/R (1/T - 1/(2T)))
        d2 = O.cell_detail(m, 2 * T, C)
        ratio = 2.0 ** 1.5 * np.exp(4000.0 / (2 * T))
        assert abs(d2["kf"][1] / d["kf"][1] / ratio - 1) < 1e-13


def test_nasa_constant_cp_closed_form():
    m = toy_mechanism()
    for T in (300.0, 999.0, 1000.0, 2500.0):
        cp, h, s, g = O.thermo(m, T)
        a1 = np.array([2.5, 3.5, 4.5])
        a6 = np.array([30000.0, 0.0, 10000.0])
        a7 = np.array([5.0, 4.0, 3.0])
        assert _rel(cp, a1) < 1e-15
        assert _rel(g, a1 * (1 - np.log(T)) + a6 / T - a7) < 1e-13


@pytest.mark.parametrize("size", ["h2air_9_21", "gri_53_325"])
def test_nasa_identities_and_continuity(size):
    """dh/dT = cp and ds/dT = cp/T on each range (central differences); h and s
    continuous at T_mid for the generated thermo; the range switch at T_mid."""
    m = synth.make_mechanism(size, seed=3)
    om = O.OracleMechanism(m)
    for T in (450.0, 800.0, 1500.0, 2600.0):
        dT = 1e-3 * T
        cp, _, _, _ = O.thermo(om, T)
        _, hp, sp, _ = O.thermo(om, T + dT)
        _, hm, sm, _ = O.thermo(om, T - dT)
        dh = ((T + dT) * hp - (T - dT) * hm) / (2 * dT)      # d(h/R)/dT
        ds = (sp - sm) / (2 * dT)                           # d(s/R)/dT
        assert _rel(dh, cp) < 1e-6
        assert _rel(ds, cp / T) < 1e-6
    tm = m.t_mid
    lo = m.nasa7[:, 0, :]
    _, h_hi, s_hi, _ = O.thermo(om, tm)                     # T >= T_mid -> high set
    # the low set evaluated at T_mid through an equivalent single-range mechanism
    m_lo = m.copy()
    m_lo.nasa7[:, 1, :] = lo
    _, h_lo, s_lo, _ = O.thermo(m_lo, tm)
    assert _rel(h_hi, h_lo) < 1e-12 and _rel(s_hi, s_lo) < 1e-12
    # just below T_mid the low set is used
    m_hi = m.copy()
    m_hi.nasa7[:, 0, :] = m.nasa7[:, 1, :]
    cp_below = O.thermo(om, tm - 1e-9)[0]
    cp_hi_below = O.thermo(m_hi, tm - 1e-9)[0]
    assert np.any(np.abs(cp_below - cp_hi_below) > 1e-6)


def test_troe_center_and_limits():
    tp = (0.6, 150.0, 2200.0, 4800.0)
    T = 1300.0
    Fc = (1 - tp[0]) * np.exp(-T / tp[1]) + tp[0] * np.exp(-T / tp[2]) + np.exp(-tp[3] / T)
    c = -0.4 - 0.67 * np.log10(Fc)
    # centre of the falloff curve: log10 Pr = -c gives F = F_cent
    assert abs(O.troe_F(tp, T, 10.0 ** (-c)) / Fc - 1) < 1e-14
    # F is between F_cent and 1 and approaches F_cent^(1/(1 + 1/0.14^2)) as Pr -> infinity
    for pr in (1e-8, 1e-2, 1.0, 1e3, 1e9):
        assert Fc - 1e-15 <= O.troe_F(tp, T, pr) <= 1.0
    lim = Fc ** (1.0 / (1.0 + (1 / 0.14) ** 2))
    e100 = abs(O.troe_F(tp, T, 1e100) / lim - 1)
    e300 = abs(O.troe_F(tp, T, 1e300) / lim - 1)
    assert e300 < e100 and e300 < 3e-3          # the approach is O(1 / log10 Pr)
    # T** absent (<= 0) drops the third term
    tp2 = (0.6, 150.0, 2200.0, 0.0)
    Fc2 = (1 - tp2[0]) * np.exp(-T / tp2[1]) + tp2[0] * np.exp(-T / tp2[2])
    c2 = -0.4 - 0.67 * np.log10(Fc2)
    assert abs(O.troe_F(tp2, T, 10.0 ** (-c2)) / Fc2 - 1) < 1e-14


def test_falloff_pressure_limits():
    """Lindemann: Pr -> infinity gives k -> k_inf; Pr -> 0 gives k -> k0 M."""
    T = 1500.0
    C = np.array([1.0e-6, 4.0e-6, 2.4e-6])
    M = C @ np.array([1.0, 2.0, 1.0])
    kinf = 1e15 / T
    for lnA0, which in ((np.log(1e40), "high"), (np.log(1e-5), "low")):
        m = toy_mechanism(synth.KIND_LINDEMANN, low1=(lnA0, 0.0, 0.0))
        kf = O.cell_detail(m, T, C)["kf"][0]
        if which == "high":
            assert abs(kf / kinf - 1) < 1e-15 * 1e6
        else:
            assert abs(kf / (np.exp(lnA0) * M) - 1) < 1e-10


# ---------------------------------------------------------------------------
# invariants on the synthetic mechanisms
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("size,n", [("h2air_9_21", 512), ("gri_53_325", 256), ("heavy_160_1000", 32)])
def test_mass_and_element_conservation(size, n):
    m = synth.make_mechanism(size, seed=2)
    kind = "dirichlet" if size == "h2air_9_21" else "mixture"
    T, P, Y = synth.make_states(m, n, seed=5, kind=kind)
    w = O.source_term(m, T, P, Y)
    mass = np.abs(w @ m.mol_weight) / (np.abs(w) @ m.mol_weight)
    assert mass.max() < 1e-12
    E = m.elem_comp.astype(float)
    el = np.abs(w @ E) / np.maximum(np.abs(w) @ E, 1e-300)
    assert el.max() < 1e-12


@pytest.mark.parametrize("size", ["h2air_9_21", "gri_53_325"])
def test_detailed_balance(size):
    """At C_k = (p_ref/RT) exp(-g_k/RT + sum_e lambda_e E_ke) every element-balanced
    reversible reaction has q_f = q_r (the lambda terms cancel by balance), third-body
    and falloff reactions included (M multiplies both directions)."""
    m = synth.make_mechanism(size, seed=4)
    om = O.OracleMechanism(m)
    rng = np.random.default_rng(11)
    for T in (900.0, 1700.0, 2600.0):
        g = O.thermo(om, T)[3]
        lam = rng.uniform(-3, 3, m.n_elements)
        C = m.p_ref / (O.R_CGS * T) * np.exp(-g + m.elem_comp @ lam)
        d = O.cell_detail(om, T, C)
        qf, qr = d["qf"], d["qr"]
        rev = m.reversible == 1
        assert np.all(np.abs(qf - qr)[rev] <= 1e-12 * qf[rev])
        scale = np.abs(m.nu_r - m.nu_f).T @ qf
        assert np.all(np.abs(d["omega"]) <= 1e-11 * np.maximum(scale, 1e-300))


@pytest.mark.parametrize("size,n", [("h2air_9_21", 300), ("gri_53_325", 100)])
def test_matrix_form_agrees_with_loop_oracle(size, n):
    m = synth.make_mechanism(size, seed=6, n_lindemann=2 if size == "gri_53_325" else 0,
                             n_irreversible=3)
    T, P, Y = synth.make_states(m, n, seed=8, kind="mixture" if size != "h2air_9_21" else "dirichlet",
                                T_range=(700.0, 2800.0))
    om = O.OracleMechanism(m)
    C = np.stack([O.concentrations(om, T[i], P[i], Y[i]) for i in range(n)])
    w_loop = O.source_term_tc(om, T, C)
    w_mat = matrix_source_term_tc(m, T, C)
    err = np.abs(w_loop - w_mat).max(1) / np.abs(w_loop).max(1)
    assert err.max() < 1e-11


def test_irreversible_reactions_have_no_reverse_rate():
    m = synth.make_mechanism("gri_53_325", seed=7, n_irreversible=20)
    T, P, Y = synth.make_states(m, 4, seed=1)
    C = O.concentrations(m, T[0], P[0], Y[0])
    d = O.cell_detail(m, T[0], C)
    irr = m.reversible == 0
    assert irr.sum() == 20
    assert np.all(d["qr"][irr] == 0.0) and np.all(d["qr"][~irr] > 0.0)


def test_zero_and_negative_mass_fractions():
    m = synth.make_mechanism("h2air_9_21", seed=1)
    T, P, Y = synth.make_states(m, 3, seed=2, kind="dirichlet")
    Y0 = Y.copy()
    Y0[:, 2] = 0.0
    Yn = Y0.copy()
    Yn[:, 2] = -1e-3                       # negative entries count as zero
    w0 = O.source_term(m, T, P, Y0)
    wn = O.source_term(m, T, P, Yn)
    assert np.all(np.isfinite(w0)) and np.array_equal(w0, wn)
    C = O.concentrations(m, T[0], P[0], Y0[0])
    d = O.cell_detail(m, T[0], C)
    has2 = m.nu_f[:, 2] > 0
    assert np.all(d["qf"][has2] == 0.0)
    assert np.all(O.source_term(m, T, P, np.zeros_like(Y)) == 0.0)


def test_threads_are_bitwise_identical(mech53):
    T, P, Y = synth.make_states(mech53, 257, seed=9)
    a = O.source_term(mech53, T, P, Y, nthreads=1)
    b = O.source_term(mech53, T, P, Y, nthreads=5)
    assert np.array_equal(a, b)


# ---------------------------------------------------------------------------
# generator
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("size", ["h2air_9_21", "gri_53_325", "heavy_160_1000"])
def test_generator_balanced_and_reproducible(size):
    a = synth.make_mechanism(size, seed=1)
    b = synth.make_mechanism(size, seed=1)
    assert a.to_json() == b.to_json()
    assert synth.Mechanism.from_json(a.to_json()).to_json() == a.to_json()
    assert np.all((a.nu_r - a.nu_f) @ a.elem_comp == 0)
    ns, nr = a.n_species, a.n_reactions
    _, _, _, n_tb, n_troe, _, _ = synth.SIZES[size]
    assert (a.kind == 1).sum() == n_tb and (a.kind == 3).sum() == n_troe
    assert np.all((a.nu_f > 0).sum(1) <= 3) and np.all(a.nu_f.sum(1) <= 3)
    assert np.all((a.nu_r > 0).sum(1) <= 3) and np.all(a.nu_r.sum(1) <= 3)
    assert not np.any((a.nu_f > 0) & (a.nu_r > 0))
    assert len({(tuple(f), tuple(r)) for f, r in zip(a.nu_f, a.nu_r)}) == nr


@pytest.mark.parametrize("size,kind,Tr,Pr", [
    ("h2air_9_21", "dirichlet", (1000.0, 2500.0), (1.0, 1.0)),
    ("gri_53_325", "mixture", (800.0, 2800.0), (1.0, 50.0)),
    ("heavy_160_1000", "mixture", (700.0, 2600.0), (1.0, 100.0)),
])
def test_log_rates_stay_in_fp32_range(size, kind, Tr, Pr):
    """Every rate of progress of the workload states has ln q < 80, so the single-
    precision paths never overflow; rates below the FP32 normal range (ln q < -87)
    carry a negligible share of omega."""
    m = synth.make_mechanism(size, seed=1)
    om = O.OracleMechanism(m)
    T, P, Y = synth.make_states(m, 64, seed=1234, kind=kind, T_range=Tr, P_atm=Pr)
    nu_abs = np.abs(m.nu_r - m.nu_f)
    worst = -np.inf
    for i in range(len(T)):
        d = O.cell_detail(om, T[i], O.concentrations(om, T[i], P[i], Y[i]))
        small = 0.0
        for q in (d["qf"], d["qr"]):
            pos = q > 0
            worst = max(worst, np.log(q[pos]).max())
            tiny = np.where(q < np.exp(-87.0), q, 0.0)
            small = np.maximum(small, nu_abs.T @ tiny)
        assert np.all(small <= 1e-12 * np.abs(d["omega"]).max())
    assert worst < 80.0


# ---------------------------------------------------------------------------
# analytic Jacobian (d omega / d(ln C, T))
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("size,kw", [("h2air_9_21", dict(n_lindemann=2, n_irreversible=3)),
                                     ("gri_53_325", dict(n_lindemann=4, n_irreversible=10))])
def test_jacobian_matches_central_differences(size, kw):
    """The oracle's analytic Jacobian against central differences of its own omega
    (step 1e-6 relative), including third-body, Lindemann, Troe and irreversible reactions,
    at states on both sides of T_mid."""
    m = synth.make_mechanism(size, seed=2, **kw)
    om = O.OracleMechanism(m)
    T, P, Y = synth.make_states(m, 6, seed=21, T_range=(700.0, 2600.0),
                                kind="dirichlet" if size == "h2air_9_21" else "mixture")
    for i in range(len(T)):
        C = O.concentrations(om, T[i], P[i], Y[i])
        J, dT = O.jacobian_tc(om, T[i], C)
        lnC = np.log(C)

        def w(T_, l_):
            return O.source_term_tc(om, [T_], np.exp(l_)[None])[0]
        Jfd = np.zeros_like(J)
        for mm in range(len(C)):
            e = np.zeros_like(lnC)
            e[mm] = 1e-6
            Jfd[:, mm] = (w(T[i], lnC + e) - w(T[i], lnC - e)) / 2e-6
        hT = 1e-6 * T[i]
        dTfd = (w(T[i] + hT, lnC) - w(T[i] - hT, lnC)) / (2 * hT)
        assert np.abs(J - Jfd).max() <= 1e-6 * np.abs(J).max()
        assert np.abs(dT - dTfd).max() <= 1e-6 * np.abs(dT).max()


def test_jacobian_detailed_balance_structure():
    """At an equilibrium composition q_f = q_r for every reaction, so d omega / d ln C
    reduces to sum_j nu_kj q_j (nu'_m - nu''_m) = -sum_j nu_kj q_j nu_mj, whose rows are
    orthogonal to the element vectors (element conservation of the linearised system)."""
    m = synth.make_mechanism("gri_53_325", seed=4)
    om = O.OracleMechanism(m)
    T = 1800.0
    g = O.thermo(om, T)[3]
    lam = np.random.default_rng(3).uniform(-2, 2, m.n_elements)
    C = m.p_ref / (O.R_CGS * T) * np.exp(-g + m.elem_comp @ lam)
    J, _ = O.jacobian_tc(om, T, C)
    q = O.cell_detail(om, T, C)["qf"]
    nu = (m.nu_r - m.nu_f).astype(float)              # [nr, ns]
    expect = -(nu.T * q) @ nu
    assert np.abs(J - expect).max() <= 1e-10 * np.abs(expect).max()
    E = m.elem_comp.astype(float)
    assert np.abs(E.T @ J).max() <= 1e-10 * np.abs(J).max()


def test_given_lnkc_reproduces_the_thermo_path(mech53):
    # with ln K_c supplied equal to the thermo value (Eq. 8), the result is unchanged; with
    # ln K_c shifted by d for one reaction, only its reverse rate scales by e^-d
    om = O.OracleMechanism(mech53)
    T, P, Y = synth.make_states(mech53, 6, seed=21)
    ref = O.source_term(om, T, P, Y)
    K = np.zeros((6, mech53.n_reactions))
    for i in range(6):
        C = O.concentrations(om, T[i], P[i], Y[i])
        K[i] = O.cell_detail(om, T[i], C)["lnKc"]
    w = O.source_term_kc(om, T, P, Y, K)
    assert np.max(np.abs(w - ref) / np.abs(ref).max(1, keepdims=True)) < 1e-14
    j = int(np.nonzero(mech53.reversible)[0][0])
    K2 = K.copy()
    K2[:, j] += 0.5
    w2 = O.source_term_kc(om, T, P, Y, K2)
    nu = (mech53.nu_r[j] - mech53.nu_f[j]).astype(float)
    for i in range(6):
        C = O.concentrations(om, T[i], P[i], Y[i])
        d = O.cell_detail(om, T[i], C)
        expect = ref[i] + nu * d["qr"][j] * (1.0 - np.exp(-0.5))
        assert np.max(np.abs(w2[i] - expect)) <= 1e-12 * np.abs(ref[i]).max()
