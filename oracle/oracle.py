"""Python access to the FP64 CPU oracle (chem_oracle.c).

TEST INFRASTRUCTURE: imported only by the tests, by the package smoke check and
by the benchmark's CPU-baseline / reference leg.  The CUDA library never
imports, links or calls it.  It computes the plain per-cell, per-reaction
definition of the net production rates (Eqs. 1-3, 5, 7, 8, 10 and Sec. 2.4),
and the constant-pressure adiabatic reactor built on them, integrated by
scipy's Radau (an implicit Runge-Kutta method of order 5, a library routine
independent of the Rosenbrock integrator of the CUDA library).

Mechanisms are any object with the array attributes of
``paper_2008_08483_gb300.synth.Mechanism``; only the data is shared.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "chem_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

R_CGS = 8.31446261815324e7


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE double, no contraction, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                        "-fno-fast-math", "-o", tmp, _SRC, "-lm", "-lpthread"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Mech(C.Structure):
    _fields_ = [("ns", C.c_int), ("nr", C.c_int),
                ("W", C.c_void_p), ("nu_f", C.c_void_p), ("nu_r", C.c_void_p),
                ("arrh", C.c_void_p), ("kind", C.c_void_p), ("rev", C.c_void_p),
                ("eff", C.c_void_p), ("arrh_low", C.c_void_p), ("troe", C.c_void_p),
                ("nasa", C.c_void_p), ("t_mid", C.c_double), ("p_ref", C.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.c_void_p
            lib.orc_thermo.argtypes = [P, C.c_double, P, P, P, P]
            lib.orc_concentrations.argtypes = [P, C.c_double, C.c_double, P, P]
            lib.orc_troe_F.argtypes = [P, C.c_double, C.c_double]
            lib.orc_troe_F.restype = C.c_double
            lib.orc_cell_detail.argtypes = [P, C.c_double, P, P, P, P, P, P, P, P, P, P]
            lib.orc_jacobian_tc.argtypes = [P, C.c_double, P, P, P, P, P]
            lib.orc_dwdC.argtypes = [P, C.c_double, P, P, P]
            lib.orc_source_term_tpy_kc.argtypes = [P, C.c_int64, P, P, P, C.c_int64, P,
                                                   C.c_int64, P, C.c_int64]
            lib.orc_source_term_tpy_kc.restype = C.c_int
            lib.orc_ode_rhs.argtypes = [P, C.c_double, P, P]
            lib.orc_ode_jac.argtypes = [P, C.c_double, P, P]
            for f in (lib.orc_source_term_tpy, lib.orc_source_term_tc):
                f.restype = C.c_int
            lib.orc_source_term_tpy.argtypes = [P, C.c_int64, P, P, P, C.c_int64, P, C.c_int64,
                                                C.c_int]
            lib.orc_source_term_tc.argtypes = [P, C.c_int64, P, P, C.c_int64, P, C.c_int64,
                                               C.c_int]
            _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


class OracleMechanism:
    """Holds contiguous copies of a mechanism's arrays and the C view of them."""

    def __init__(self, mech):
        self.ns = int(mech.nu_f.shape[1])
        self.nr = int(mech.nu_f.shape[0])
        self._keep = dict(
            W=np.ascontiguousarray(mech.mol_weight, np.float64),
            nu_f=np.ascontiguousarray(mech.nu_f, np.int32),
            nu_r=np.ascontiguousarray(mech.nu_r, np.int32),
            arrh=np.ascontiguousarray(mech.arrh, np.float64),
            kind=np.ascontiguousarray(mech.kind, np.int32),
            rev=np.ascontiguousarray(mech.reversible, np.int32),
            eff=np.ascontiguousarray(mech.eff, np.float64),
            arrh_low=np.ascontiguousarray(mech.arrh_low, np.float64),
            troe=np.ascontiguousarray(mech.troe, np.float64),
            nasa=np.ascontiguousarray(mech.nasa7, np.float64),
        )
        k = self._keep
        self.c = _Mech(self.ns, self.nr, *(_ptr(k[n]).value for n in (
            "W", "nu_f", "nu_r", "arrh", "kind", "rev", "eff", "arrh_low", "troe", "nasa")),
            float(mech.t_mid), float(mech.p_ref))
        self.ref = C.byref(self.c)


def _om(mech):
    return mech if isinstance(mech, OracleMechanism) else OracleMechanism(mech)


def default_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def thermo(mech, T: float):
    """(cp/R, h/RT, s/R, g/RT) per species at temperature T (NASA-7, Eq. 10)."""
    om = _om(mech)
    out = [np.zeros(om.ns) for _ in range(4)]
    _load().orc_thermo(om.ref, float(T), *(_ptr(a) for a in out))
    return tuple(out)


def concentrations(mech, T: float, P: float, Y) -> np.ndarray:
    om = _om(mech)
    Y = np.ascontiguousarray(Y, np.float64)
    out = np.zeros(om.ns)
    _load().orc_concentrations(om.ref, float(T), float(P), _ptr(Y), _ptr(out))
    return out


def troe_F(troe_params, T: float, Pr: float) -> float:
    tp = np.ascontiguousarray(troe_params, np.float64)
    return float(_load().orc_troe_F(_ptr(tp), float(T), float(Pr)))


def cell_detail(mech, T: float, C_):
    """Per-reaction intermediates for one cell at (T, C): dict of arrays."""
    om = _om(mech)
    Cc = np.ascontiguousarray(C_, np.float64)
    names = ("lnkf", "lnKc", "M", "kf", "kr", "qf", "qr")
    out = {n: np.zeros(om.nr) for n in names}
    out["omega"] = np.zeros(om.ns)
    g = np.zeros(om.ns)
    _load().orc_cell_detail(om.ref, float(T), _ptr(Cc), _ptr(g),
                            *(_ptr(out[n]) for n in names), _ptr(out["omega"]))
    return out


def source_term(mech, T, P, Y, nthreads: int | None = None) -> np.ndarray:
    """omega [n, ns] (mol/(cm^3 s)) from T [n] (K), P [n] (dyn/cm^2), Y [n, ns]."""
    om = _om(mech)
    T = np.ascontiguousarray(T, np.float64)
    P = np.ascontiguousarray(P, np.float64)
    Y = np.ascontiguousarray(Y, np.float64)
    n = T.shape[0]
    out = np.zeros((n, om.ns))
    rc = _load().orc_source_term_tpy(om.ref, n, _ptr(T), _ptr(P), _ptr(Y), Y.shape[1],
                                     _ptr(out), om.ns, nthreads or default_threads())
    if rc != 0:
        raise RuntimeError("oracle source term failed")
    return out


def source_term_tc(mech, T, Cc, nthreads: int | None = None) -> np.ndarray:
    """omega [n, ns] from T [n] and concentrations C [n, ns] (mol/cm^3)."""
    om = _om(mech)
    T = np.ascontiguousarray(T, np.float64)
    Cc = np.ascontiguousarray(Cc, np.float64)
    n = T.shape[0]
    out = np.zeros((n, om.ns))
    rc = _load().orc_source_term_tc(om.ref, n, _ptr(T), _ptr(Cc), Cc.shape[1], _ptr(out),
                                    om.ns, nthreads or default_threads())
    if rc != 0:
        raise RuntimeError("oracle source term failed")
    return out


def jacobian_tc(mech, T: float, C_):
    """Analytic d omega / d ln C [ns, ns] and d omega / dT [ns] at (T, C)."""
    om = _om(mech)
    Cc = np.ascontiguousarray(C_, np.float64)
    J = np.zeros((om.ns, om.ns))
    dT = np.zeros(om.ns)
    h = np.zeros(om.ns)
    g = np.zeros(om.ns)
    _load().orc_jacobian_tc(om.ref, float(T), _ptr(Cc), _ptr(h), _ptr(g), _ptr(J), _ptr(dT))
    return J, dT


def dwdC(mech, T: float, C_):
    """d omega / dC [ns, ns] and d omega / dT at fixed C [ns] (direct mass-action form)."""
    om = _om(mech)
    Cc = np.ascontiguousarray(C_, np.float64)
    J = np.zeros((om.ns, om.ns))
    dT = np.zeros(om.ns)
    _load().orc_dwdC(om.ref, float(T), _ptr(Cc), _ptr(J), _ptr(dT))
    return J, dT


def ode_rhs(mech, P: float, y):
    """Right-hand side of the constant-pressure adiabatic reactor, y = (T, Y_1..Y_ns)."""
    om = _om(mech)
    y = np.ascontiguousarray(y, np.float64)
    f = np.zeros(om.ns + 1)
    _load().orc_ode_rhs(om.ref, float(P), _ptr(y), _ptr(f))
    return f


def ode_jac(mech, P: float, y):
    """Analytic Jacobian [ns+1, ns+1] of ode_rhs (row: component of f, column: of y)."""
    om = _om(mech)
    y = np.ascontiguousarray(y, np.float64)
    J = np.zeros((om.ns + 1, om.ns + 1))
    _load().orc_ode_jac(om.ref, float(P), _ptr(y), _ptr(J))
    return J


def integrate_reactor(mech, T0: float, P: float, Y0, t_end: float, rtol: float = 1e-10,
                      atol: float = 1e-20, ign_dT: float = 400.0, t_eval=None):
    """Constant-pressure adiabatic reactor from (T0, Y0) to t_end with scipy Radau on the
    oracle's right-hand side and analytic Jacobian.  The ignition delay is the first time at
    which T reaches T0 + ign_dT (an event located on Radau's dense output); NaN if never."""
    from scipy.integrate import solve_ivp

    om = _om(mech)
    y0 = np.concatenate([[float(T0)], np.asarray(Y0, np.float64)])
    target = float(T0) + ign_dT

    def ev(t, y):
        return y[0] - target
    ev.direction = 1.0
    sol = solve_ivp(lambda t, y: ode_rhs(om, P, y), (0.0, float(t_end)), y0, method="Radau",
                    jac=lambda t, y: ode_jac(om, P, y), rtol=rtol, atol=atol, events=ev,
                    t_eval=t_eval)
    if sol.status != 0:
        raise RuntimeError("oracle reactor integration failed: " + str(sol.message))
    t_ign = float(sol.t_events[0][0]) if len(sol.t_events[0]) else float("nan")
    return dict(y_end=sol.y[:, -1].copy(), t_ign=t_ign, nfev=int(sol.nfev),
                njev=int(sol.njev), nsteps=int(len(sol.t) - 1) if t_eval is None else -1, sol=sol)


def source_term_kc(mech, T, P, Y, lnKc) -> np.ndarray:
    """omega [n, ns] with the ln K_c of every cell and reaction given, lnKc [n, nr]."""
    om = _om(mech)
    T = np.ascontiguousarray(T, np.float64)
    P = np.ascontiguousarray(P, np.float64)
    Y = np.ascontiguousarray(Y, np.float64)
    K = np.ascontiguousarray(lnKc, np.float64)
    out = np.zeros((T.shape[0], om.ns))
    if _load().orc_source_term_tpy_kc(om.ref, T.shape[0], _ptr(T), _ptr(P), _ptr(Y), Y.shape[1],
                                      _ptr(K), K.shape[1], _ptr(out), om.ns) != 0:
        raise RuntimeError("oracle source term failed")
    return out
