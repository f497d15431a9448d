"""Toy mechanisms whose constant-pressure reactor has a closed-form solution or invariant.

Test inputs only: the mechanisms are built by hand and the closed forms are derived from the
reactor equations (constant pressure, adiabatic), not from either implementation.
"""
import numpy as np
from scipy.optimize import brentq

from paper_2008_08483_gb300 import synth

R = synth.R_CGS


def _mech(name, species, comp, W, nu_f, nu_r, arrh, rev, nasa_rows):
    ns, nr = len(species), len(nu_f)
    nasa = np.zeros((ns, 2, 7))
    for k, row in enumerate(nasa_rows):
        nasa[k, 0] = row
        nasa[k, 1] = row
    return synth.Mechanism(
        name=name, elements=["X"], species=list(species),
        elem_comp=np.array(comp, np.int32).reshape(ns, 1), mol_weight=np.array(W, float),
        nu_f=np.array(nu_f, np.int32), nu_r=np.array(nu_r, np.int32),
        arrh=np.array(arrh, float), kind=np.zeros(nr, np.int32),
        reversible=np.array(rev, np.int32), eff=np.ones((nr, ns)), arrh_low=np.zeros((nr, 3)),
        troe=np.zeros((nr, 4)), nasa7=nasa, t_mid=1000.0, p_ref=1e6)


def isomerisation(k=1.0, da7=1.0):
    """A <=> B with equal composition, weight and enthalpy: T and rho stay constant and
    K_c = exp(a7_B - a7_A) = exp(da7), so Y_A relaxes exponentially."""
    rows = [[3.5, 0, 0, 0, 0, -1000.0, 3.0], [3.5, 0, 0, 0, 0, -1000.0, 3.0 + da7]]
    return _mech("iso", ["A", "B"], [2, 2], [20.0, 20.0], [[1, 0]], [[0, 1]],
                 [[np.log(k), 0.0, 0.0]], [1], rows)


def isomerisation_exact(k, da7, YA0, t):
    kr = k / np.exp(da7)
    yeq = kr / (k + kr)
    return yeq + (YA0 - yeq) * np.exp(-(k + kr) * np.asarray(t, float))


def dimerisation(k=1e12):
    """2 A -> B (irreversible), B with twice A's weight and NASA coefficients a1..a6: the
    enthalpy and heat capacity of the mixture do not change, so T is constant, while the
    mass density changes with the mean molecular weight at constant pressure."""
    a = [3.0, 1e-4, 0.0, 0.0, 0.0, -500.0, 2.0]
    b = [2 * x for x in a[:6]] + [1.0]
    return _mech("dimer", ["A", "B"], [1, 2], [10.0, 20.0], [[2, 0]], [[0, 1]],
                 [[np.log(k), 0.0, 0.0]], [0], [a, b])


def dimerisation_exact(k, T, P, t, YA0=1.0):
    """Y_A(t): dY/dt = -K Y^2 / (1 + Y), K = 4 k P / (R T) (W_A = 10), hence
    (ln Y - 1/Y) - (ln Y0 - 1/Y0) = -K t."""
    K = 4.0 * k * P / (R * T)
    G = lambda y: np.log(y) - 1.0 / y
    out = []
    for tt in np.atleast_1d(t):
        target = G(YA0) - K * tt
        out.append(YA0 if tt == 0 else brentq(lambda y: G(y) - target, 1e-300, YA0, xtol=1e-300,
                                                rtol=1e-15, maxiter=500))
    return np.array(out)


def exothermic(lnA=12.0, EoR=10000.0, dh=20000.0):
    """A -> B (irreversible), isomers with the same constant cp/R = 3.5 and h_A - h_B = R dh
    (erg/mol): adiabatic at constant pressure, T = T0 + (dh / 3.5) (Y_A0 - Y_A)."""
    rows = [[3.5, 0, 0, 0, 0, dh, 3.0], [3.5, 0, 0, 0, 0, 0.0, 3.0]]
    return _mech("exo", ["A", "B"], [2, 2], [20.0, 20.0], [[1, 0]], [[0, 1]],
                 [[lnA, 0.0, EoR]], [0], rows)
