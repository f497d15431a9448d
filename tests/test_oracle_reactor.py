"""Pins of the oracle's constant-pressure adiabatic reactor (right-hand side, Jacobian, and
the scipy Radau integration built on them) against closed forms, invariants and finite
differences."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2008_08483_gb300 import synth

import reactor_toys as toys

R = synth.R_CGS


def _states(mech, n, seed):
    T, P, Y, _ = synth.make_ignition_states(mech, n, seed=seed)
    rng = np.random.default_rng(seed)
    # partially burnt states with trace radicals, and exact zeros
    Yb = Y * (1 - 0.3) + 0.3 * rng.dirichlet(np.full(mech.n_species, 0.3), n)
    Yb[:, rng.integers(0, mech.n_species, 5)] = 0.0
    return np.concatenate([T, T + 600]), np.concatenate([P, P]), np.concatenate([Y, Yb])


def _fd_jac(om, P, y):
    n = len(y)
    J = np.zeros((n, n))
    for c in range(n):
        h = 1e-4 if c == 0 else 1e-6 * max(abs(y[c]), 1e-3)
        yp, ym = y.copy(), y.copy()
        yp[c] += h
        ym[c] -= h
        J[:, c] = (O.ode_rhs(om, P, yp) - O.ode_rhs(om, P, ym)) / (2 * h)
    return J


@pytest.mark.parametrize("size", ["h2air_9_21", "gri_53_325"])
def test_reactor_jacobian_matches_central_differences(size):
    m = synth.make_mechanism(size, seed=1)
    om = O.OracleMechanism(m)
    T, P, Y = _states(m, 3, seed=5)
    for i in range(len(T)):
        y = np.concatenate([[T[i]], Y[i]])
        J = O.ode_jac(om, P[i], y)
        Jfd = _fd_jac(om, P[i], y)
        # per column relative to the column's scale (T and Y columns differ by 1e3-1e9)
        for c in range(len(y)):
            sc = max(np.max(np.abs(Jfd[:, c])), 1e-300)
            assert np.max(np.abs(J[:, c] - Jfd[:, c])) / sc < 2e-5, (i, c)


def test_dwdC_matches_log_jacobian_away_from_zero():
    # d omega/dC_m = (d omega/d ln C_m) / C_m where C_m > 0: the direct and logarithmic forms
    m = synth.make_mechanism("gri_53_325", seed=1)
    om = O.OracleMechanism(m)
    T, P, Y = _states(m, 2, seed=9)
    for i in range(2):
        C = O.concentrations(om, T[i], P[i], np.maximum(Y[i], 1e-12))
        Jd, dTd = O.dwdC(om, T[i], C)
        Jl, dTl = O.jacobian_tc(om, T[i], C)
        assert np.max(np.abs(Jd * C[None, :] - Jl)) / np.max(np.abs(Jl)) < 1e-12
        assert np.max(np.abs(dTd - dTl)) / np.max(np.abs(dTl)) < 1e-12


@pytest.mark.parametrize("size", ["h2air_9_21", "gri_53_325", "heavy_160_1000"])
def test_reactor_rhs_invariants(size):
    # sum_k dY_k/dt = 0, elements conserved, and d/dt sum_k Y_k H_k / W_k = 0 (adiabatic,
    # constant pressure): sum_k (H_k / W_k) dY_k/dt + c_p dT/dt = 0
    m = synth.make_mechanism(size, seed=1)
    om = O.OracleMechanism(m)
    T, P, Y = _states(m, 3, seed=3)
    for i in range(len(T)):
        y = np.concatenate([[T[i]], Y[i]])
        f = O.ode_rhs(om, P[i], y)
        fY = f[1:]
        sc = np.max(np.abs(fY))
        assert abs(fY.sum()) / sc < 1e-12
        el = (fY / m.mol_weight) @ m.elem_comp
        assert np.max(np.abs(el)) / np.max(np.abs(fY / m.mol_weight)) < 1e-12
        cpR, hRT, _, _ = O.thermo(om, T[i])
        H = R * T[i] * hRT
        cp = R * np.sum(Y[i] * cpR / m.mol_weight)
        terms = np.concatenate([H / m.mol_weight * fY, [cp * f[0]]])
        assert abs(terms.sum()) / np.max(np.abs(terms)) < 1e-11


def test_isomerisation_closed_form():
    k, da7 = 50.0, 1.0
    m = toys.isomerisation(k, da7)
    om = O.OracleMechanism(m)
    t_eval = np.linspace(0, 0.05, 11)
    r = O.integrate_reactor(om, 1200.0, 2e6, [0.9, 0.1], 0.05, t_eval=t_eval)
    ya = r["sol"].y[1]
    assert np.max(np.abs(ya - toys.isomerisation_exact(k, da7, 0.9, t_eval))) < 1e-9
    assert np.max(np.abs(r["sol"].y[0] - 1200.0)) < 1e-9


def test_dimerisation_closed_form():
    # density changes with the mean molecular weight at constant pressure
    k, T, P = 1e12, 1500.0, 3e6
    m = toys.dimerisation(k)
    om = O.OracleMechanism(m)
    t_eval = np.array([0.0, 1e-8, 1e-7, 1e-6, 1e-5])
    r = O.integrate_reactor(om, T, P, [1.0, 0.0], 1e-5, t_eval=t_eval)
    exact = toys.dimerisation_exact(k, T, P, t_eval)
    assert np.max(np.abs(r["sol"].y[1] - exact) / exact) < 1e-7
    assert np.max(np.abs(r["sol"].y[0] - T)) < 1e-7


def test_exothermic_temperature_invariant():
    dh = 20000.0
    m = toys.exothermic(lnA=14.0, EoR=10000.0, dh=dh)
    om = O.OracleMechanism(m)
    t_eval = np.linspace(0, 2e-3, 41)
    r = O.integrate_reactor(om, 1000.0, 1e6, [1.0, 0.0], 2e-3, t_eval=t_eval)
    T, ya = r["sol"].y[0], r["sol"].y[1]
    assert ya[-1] < 0.5      # the reaction ran (thermal runaway)
    assert np.max(np.abs(T - (1000.0 + dh / 3.5 * (1.0 - ya)))) < 1e-6
    # the ignition event (T0 + 400 K) lies on the trajectory
    assert np.isfinite(r["t_ign"]) and 0 < r["t_ign"] < 2e-3


def test_reactor_reaches_equilibrium_with_invariants():
    m = synth.make_mechanism("h2air_9_21", seed=1)
    om = O.OracleMechanism(m)
    T, P, Y, _ = synth.make_ignition_states(m, 1, seed=11)
    r = O.integrate_reactor(om, T[0], P[0], Y[0], 1.0, rtol=1e-10, atol=1e-20)
    y = r["y_end"]
    assert abs(y[1:].sum() - 1.0) < 1e-10
    el0 = (Y[0] / m.mol_weight) @ m.elem_comp
    el1 = (y[1:] / m.mol_weight) @ m.elem_comp
    assert np.max(np.abs(el1 - el0) / el0) < 1e-9
    _, hRT0, _, _ = O.thermo(om, T[0])
    _, hRT1, _, _ = O.thermo(om, y[0])
    h0 = np.sum(Y[0] * R * T[0] * hRT0 / m.mol_weight)
    h1 = np.sum(y[1:] * R * y[0] * hRT1 / m.mol_weight)
    assert abs(h1 - h0) / abs(R * T[0] * np.max(np.abs(hRT0)) / m.mol_weight.min()) < 1e-8
    # detailed balance at the end state: q_f = q_r for every reversible reaction
    rho = P[0] / (R * y[0] * np.sum(y[1:] / m.mol_weight))
    C = rho * y[1:] / m.mol_weight
    d = O.cell_detail(om, y[0], C)
    big = d["qf"] > 1e-30 * d["qf"].max()
    assert np.max(np.abs(d["qf"] - d["qr"])[big] / d["qf"][big]) < 1e-5
