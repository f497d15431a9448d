"""Seeded synthetic chemical mechanisms and cell states.

This module only *constructs inputs*: a mechanism descriptor (species, element
compositions, stoichiometry, Arrhenius / third-body / falloff parameters and
two-range NASA-7 thermo) and batches of cell states (T, P, Y).  It evaluates no
rate, equilibrium constant or production rate; both the CPU oracle and the CUDA
path consume what it returns.

The mechanisms stand in for the paper's H2/air, CH4 and UCSD mechanisms
(Table 1), which are not available.  Their structure follows the paper: a
reversible mechanism (Eq. 1) with third-body and Troe falloff reactions
(Sec. 2.4) and NASA-7 polynomials with a common switch temperature
(Eq. 10, "usually 1000 K").  Parameter ranges: ln A ~ U[20, 35] (cgs units),
b ~ U[-2, 2], E/R ~ U[0, 25000] K, third-body efficiencies U[0.5, 5] on a
random 3-6 species subset.

Two pieces of thermo construction live here because the generator must emit
consistent NASA-7 sets: the quartic cp fit on each range and the integration
constants (a6, a7) that make h and s continuous at T_mid.  They are the
standard NASA-7 antiderivatives applied to the generator's own targets; the
oracle's tests check continuity and dh/dT = cp independently.
"""
from __future__ import annotations

import itertools
import json
from dataclasses import dataclass, field

import numpy as np

R_CGS = 8.31446261815324e7        # erg / (mol K)
P_ATM = 1.01325e6                 # dyn / cm^2
P_BAR = 1.0e6                     # dyn / cm^2 (the paper's p_ref, Eq. 8)

ATOMIC_WEIGHT = {"H": 1.008, "C": 12.011, "N": 14.007, "O": 15.999, "Ar": 39.948}

KIND_ELEMENTARY, KIND_THIRD_BODY, KIND_LINDEMANN, KIND_TROE = 0, 1, 2, 3


@dataclass
class Mechanism:
    """Plain-array mechanism descriptor (cgs units).

    Stoichiometry is stored reaction-major: ``nu_f[j, k]`` is the reactant
    coefficient of species k in reaction j (the paper's nu'_{kj}, Eq. 1) and
    ``nu_r[j, k]`` the product coefficient (nu''_{kj}).
    """

    name: str
    elements: list
    species: list
    elem_comp: np.ndarray          # [ns, ne] int32 atom counts
    mol_weight: np.ndarray         # [ns] g/mol
    nu_f: np.ndarray               # [nr, ns] int32
    nu_r: np.ndarray               # [nr, ns] int32
    arrh: np.ndarray               # [nr, 3] ln A (cgs), b, E/R [K]
    kind: np.ndarray               # [nr] int32: 0 elementary, 1 third body, 2 Lindemann, 3 Troe
    reversible: np.ndarray         # [nr] int32
    eff: np.ndarray                # [nr, ns] third-body efficiencies (1 = default)
    arrh_low: np.ndarray           # [nr, 3] low-pressure Arrhenius for falloff reactions
    troe: np.ndarray               # [nr, 4] alpha, T***, T*, T** (T** <= 0: term absent)
    nasa7: np.ndarray              # [ns, 2, 7] coefficient sets: [:,0] T < t_mid, [:,1] T >= t_mid
    t_mid: float = 1000.0
    p_ref: float = P_BAR
    seed: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def n_species(self) -> int:
        return len(self.species)

    @property
    def n_reactions(self) -> int:
        return int(self.nu_f.shape[0])

    @property
    def n_elements(self) -> int:
        return len(self.elements)

    def species_index(self, name: str) -> int:
        return self.species.index(name)

    # -- text format -------------------------------------------------------
    _ARRAYS = ("elem_comp", "mol_weight", "nu_f", "nu_r", "arrh", "kind", "reversible",
               "eff", "arrh_low", "troe", "nasa7")

    def to_json(self) -> str:
        d = {"name": self.name, "elements": self.elements, "species": self.species,
             "t_mid": self.t_mid, "p_ref": self.p_ref, "seed": self.seed, "meta": self.meta}
        for a in self._ARRAYS:
            arr = getattr(self, a)
            d[a] = {"dtype": str(arr.dtype), "shape": list(arr.shape),
                    "data": [float.hex(float(x)) if arr.dtype.kind == "f" else int(x)
                             for x in arr.ravel()]}
        return json.dumps(d)

    @classmethod
    def from_json(cls, text: str) -> "Mechanism":
        d = json.loads(text)
        kw = {k: d[k] for k in ("name", "elements", "species", "t_mid", "p_ref", "seed", "meta")}
        for a in cls._ARRAYS:
            e = d[a]
            vals = [float.fromhex(x) if isinstance(x, str) else x for x in e["data"]]
            kw[a] = np.array(vals, dtype=e["dtype"]).reshape(e["shape"])
        return cls(**kw)

    def copy(self) -> "Mechanism":
        return Mechanism.from_json(self.to_json())


# ---------------------------------------------------------------------------
# species
# ---------------------------------------------------------------------------

def _formula(comp: dict) -> str:
    out = []
    for el in ("C", "H", "O", "N", "Ar"):
        n = comp.get(el, 0)
        if n:
            out.append(el if n == 1 else f"{el}{n}")
    return "".join(out)


SIZES = {
    # key: (elements, n_species, n_reactions, n_third_body, n_troe, anchors, pool limits)
    "h2air_9_21": (["H", "O", "N"], 9, 21, 5, 0,
                   [{"H": 2}, {"O": 2}, {"H": 2, "O": 1}, {"N": 2}, {"H": 1}, {"O": 1},
                    {"H": 1, "O": 1}],
                   {"C": 0, "H": 3, "O": 2, "N": 2, "atoms": 4}),
    "gri_53_325": (["C", "H", "O", "N", "Ar"], 53, 325, 30, 25,
                   [{"C": 1, "H": 4}, {"O": 2}, {"N": 2}, {"H": 2, "O": 1}, {"C": 1, "O": 2},
                    {"C": 1, "O": 1}, {"H": 2}, {"Ar": 1}, {"H": 1}, {"O": 1}, {"H": 1, "O": 1}],
                   {"C": 3, "H": 8, "O": 2, "N": 1, "atoms": 10}),
    "heavy_160_1000": (["C", "H", "O", "N"], 160, 1000, 90, 75,
                       [{"C": 7, "H": 16}, {"O": 2}, {"N": 2}, {"H": 2, "O": 1}, {"C": 1, "O": 2},
                        {"C": 1, "O": 1}, {"H": 2}, {"H": 1}, {"O": 1}, {"H": 1, "O": 1}],
                       {"C": 8, "H": 18, "O": 3, "N": 1, "atoms": 24}),
}

# formation enthalpy targets h_f(298)/R [K] for the anchor species (generic magnitudes:
# element references 0, water/CO2/CO strongly negative, atoms and radicals positive)
_ANCHOR_HF = {"H2": 0.0, "O2": 0.0, "N2": 0.0, "Ar": 0.0, "H2O": -29000.0, "CO2": -47300.0,
              "CO": -13300.0, "CH4": -9000.0, "C7H16": -22500.0, "H": 26000.0, "O": 30000.0,
              "HO": 4500.0}


def _species_pool(elements, lim):
    pool = []
    rng_c = range(lim["C"] + 1) if "C" in elements else [0]
    rng_h = range(lim["H"] + 1)
    rng_o = range(lim["O"] + 1)
    rng_n = range(lim["N"] + 1) if "N" in elements else [0]
    for c, h, o, n in itertools.product(rng_c, rng_h, rng_o, rng_n):
        tot = c + h + o + n
        if tot == 0 or tot > lim["atoms"]:
            continue
        comp = {k: v for k, v in (("C", c), ("H", h), ("O", o), ("N", n)) if v}
        pool.append(comp)
    return pool


def _pick_species(rng, elements, n_species, anchors, lim):
    chosen = [dict(a) for a in anchors]
    keys = {_formula(a) for a in chosen}
    pool = [c for c in _species_pool(elements, lim) if _formula(c) not in keys]
    # prefer small molecules (radicals and stable small species) for half of the picks
    small = [c for c in pool if sum(c.values()) <= 4]
    large = [c for c in pool if sum(c.values()) > 4]
    need = n_species - len(chosen)
    n_small = min(len(small), need // 2 + need % 2)
    idx_s = rng.choice(len(small), size=n_small, replace=False)
    picks = [small[i] for i in idx_s]
    rest = [c for i, c in enumerate(small) if i not in set(idx_s.tolist())] + large
    idx_l = rng.choice(len(rest), size=need - n_small, replace=False)
    picks += [rest[i] for i in idx_l]
    chosen += picks
    return chosen


# ---------------------------------------------------------------------------
# thermo construction (NASA-7 from cp / h / s targets)
# ---------------------------------------------------------------------------

def _fit_cp(cp_fun, t_lo, t_hi):
    """Least-squares quartic in T for cp/R on [t_lo, t_hi]; returns a1..a5."""
    t = np.linspace(t_lo, t_hi, 200)
    tau = t / 1000.0
    V = np.vander(tau, 5, increasing=True)
    b, *_ = np.linalg.lstsq(V, cp_fun(t), rcond=None)
    return b / (1000.0 ** np.arange(5))


def _h_over_r_poly(a, T):
    # integral of cp/R dT without the integration constant
    return a[0] * T + a[1] * T**2 / 2 + a[2] * T**3 / 3 + a[3] * T**4 / 4 + a[4] * T**5 / 5


def _s_over_r_poly(a, T):
    # integral of cp/(R T) dT without the integration constant
    return a[0] * np.log(T) + a[1] * T + a[2] * T**2 / 2 + a[3] * T**3 / 3 + a[4] * T**4 / 4


def _nasa_for_species(rng, comp, name, t_mid):
    n_atoms = sum(comp.values())
    if n_atoms == 1:
        cp0, cpinf = 2.5, 2.5 + rng.uniform(0.0, 0.3)
    elif n_atoms == 2:
        cp0, cpinf = 3.5, 4.5
    else:
        cp0, cpinf = 4.0 + 0.5 * (n_atoms - 3), 3.0 * n_atoms - 2.0
    theta = rng.uniform(800.0, 2000.0)
    # +-5 % perturbation of the cp targets around the small-molecule shapes
    cp0 *= rng.uniform(0.95, 1.05)
    cpinf *= rng.uniform(0.95, 1.05)
    theta *= rng.uniform(0.95, 1.05)

    def cp_fun(t):
        u2 = (t / theta) ** 2
        return cp0 + (cpinf - cp0) * u2 / (1.0 + u2)

    lo = _fit_cp(cp_fun, 300.0, t_mid)
    hi = _fit_cp(cp_fun, t_mid, 5000.0)
    if name in _ANCHOR_HF:
        hf = _ANCHOR_HF[name] * rng.uniform(0.95, 1.05)
    elif n_atoms == 1:
        hf = rng.uniform(20000.0, 60000.0)
    else:
        hf = rng.uniform(-50000.0, 60000.0) * (0.5 if n_atoms > 6 else 1.0)
    s298 = float(np.clip(15.0 + 2.0 * n_atoms + rng.uniform(-2.0, 2.0), 15.0, 35.0 + n_atoms))
    T0 = 298.15
    a6_lo = hf - _h_over_r_poly(lo, T0)
    a7_lo = s298 - _s_over_r_poly(lo, T0)
    h_mid = _h_over_r_poly(lo, t_mid) + a6_lo
    s_mid = _s_over_r_poly(lo, t_mid) + a7_lo
    a6_hi = h_mid - _h_over_r_poly(hi, t_mid)
    a7_hi = s_mid - _s_over_r_poly(hi, t_mid)
    out = np.zeros((2, 7))
    out[0, :5], out[0, 5], out[0, 6] = lo, a6_lo, a7_lo
    out[1, :5], out[1, 5], out[1, 6] = hi, a6_hi, a7_hi
    return out, hf


# ---------------------------------------------------------------------------
# reactions
# ---------------------------------------------------------------------------

def _enumerate_sides(comp):
    """All reaction sides with 1-3 distinct species, coefficients in {1, 2}, order <= 3.

    Returns (species [n,3] (-1 pad), coeffs [n,3], order [n], element vectors [n, ne])."""
    ns = comp.shape[0]
    sp, nu = [], []
    for k in range(ns):
        sp += [(k, -1, -1), (k, -1, -1)]
        nu += [(1, 0, 0), (2, 0, 0)]
    pairs = np.array(list(itertools.combinations(range(ns), 2)), dtype=np.int64).reshape(-1, 2)
    for c in ((1, 1), (2, 1), (1, 2)):
        sp.append(np.column_stack([pairs, -np.ones(len(pairs), np.int64)]))
        nu.append(np.tile(np.array([c[0], c[1], 0]), (len(pairs), 1)))
    sp_single = np.array(sp[: 2 * ns], dtype=np.int64)
    nu_single = np.array(nu[: 2 * ns], dtype=np.int64)
    sp_rest = np.concatenate(sp[2 * ns:]) if len(sp) > 2 * ns else np.zeros((0, 3), np.int64)
    nu_rest = np.concatenate(nu[2 * ns:]) if len(nu) > 2 * ns else np.zeros((0, 3), np.int64)
    trip = np.array(list(itertools.combinations(range(ns), 3)), dtype=np.int64).reshape(-1, 3)
    SP = np.concatenate([sp_single, sp_rest, trip])
    NU = np.concatenate([nu_single, nu_rest, np.ones_like(trip)])
    ORD = NU.sum(1)
    compz = np.vstack([comp, np.zeros((1, comp.shape[1]), comp.dtype)])
    EV = (compz[SP] * NU[:, :, None]).sum(1)
    return SP, NU, ORD, EV


def _side_dict(sp, nu):
    return {int(s): int(n) for s, n in zip(sp, nu) if s >= 0}


class _ReactionDrawer:
    def __init__(self, rng, comp):
        self.rng = rng
        self.SP, self.NU, self.ORD, EV = _enumerate_sides(comp)
        _, self.bucket = np.unique(EV, axis=0, return_inverse=True)
        self.bucket = self.bucket.ravel()
        order = np.argsort(self.bucket, kind="stable")
        self.sorted_idx = order
        bsorted = self.bucket[order]
        nb = int(bsorted.max()) + 1
        self.bstart = np.searchsorted(bsorted, np.arange(nb))
        self.bend = np.searchsorted(bsorted, np.arange(nb), side="right")
        self.by_order = {o: np.nonzero(self.ORD == o)[0] for o in (1, 2, 3)}
        self.seen = set()

    def _partners(self, s1, o2):
        b = self.bucket[s1]
        cand = self.sorted_idx[self.bstart[b]:self.bend[b]]
        cand = cand[self.ORD[cand] == o2]
        sp1 = set(int(x) for x in self.SP[s1] if x >= 0)
        ok = [c for c in cand if c != s1 and not (sp1 & set(int(x) for x in self.SP[c] if x >= 0))]
        return ok

    def draw(self, o1, o2, must_contain=None, tries=400):
        for _ in range(tries):
            pool = self.by_order[o1]
            if must_contain is not None:
                pool = pool[(self.SP[pool] == must_contain).any(1)]
                if len(pool) == 0:
                    return None
            s1 = int(self.rng.choice(pool))
            ok = self._partners(s1, o2)
            if not ok:
                continue
            s2 = int(self.rng.choice(ok))
            key = frozenset((s1, s2))
            if key in self.seen:
                continue
            self.seen.add(key)
            return (_side_dict(self.SP[s1], self.NU[s1]), _side_dict(self.SP[s2], self.NU[s2]))
        return None


_PLAIN_TYPES = [((2, 2), 0.62), ((1, 2), 0.17), ((2, 3), 0.09), ((1, 1), 0.03), ((1, 3), 0.05),
                ((3, 3), 0.04)]


def make_mechanism(size: str = "gri_53_325", seed: int = 1, n_lindemann: int = 0,
                   n_irreversible: int = 0) -> Mechanism:
    """Build a seeded synthetic mechanism of one of the sizes in ``SIZES``.

    ``n_lindemann`` falloff reactions without a Troe function and ``n_irreversible``
    irreversible reactions can be added for coverage; the sized workloads use none.
    """
    elements, ns, nr, n_tb, n_troe, anchors, lim = SIZES[size]
    rng = np.random.default_rng(np.random.PCG64(seed))
    comps = _pick_species(rng, elements, ns, anchors, lim)
    names = [_formula(c) for c in comps]
    ne = len(elements)
    comp = np.array([[c.get(e, 0) for e in elements] for c in comps], dtype=np.int32)
    W = np.array([sum(ATOMIC_WEIGHT[e] * c.get(e, 0) for e in elements) for c in comps])
    t_mid = 1000.0
    nasa = np.zeros((ns, 2, 7))
    hf = np.zeros(ns)
    for k, (c, nm) in enumerate(zip(comps, names)):
        nasa[k], hf[k] = _nasa_for_species(rng, c, nm, t_mid)

    drawer = _ReactionDrawer(rng, comp)
    reactions = []          # (reactants, products, kind)
    n_fall = n_troe + n_lindemann
    kinds = [KIND_TROE] * n_troe + [KIND_LINDEMANN] * n_lindemann + [KIND_THIRD_BODY] * n_tb
    types = [t for t, _ in _PLAIN_TYPES]
    probs = np.array([p for _, p in _PLAIN_TYPES])
    probs /= probs.sum()

    def draw_any():
        for _ in range(200):
            o1, o2 = types[rng.choice(len(types), p=probs)]
            r = drawer.draw(o1, o2, tries=50)
            if r is not None:
                return r
        raise RuntimeError(f"cannot draw {nr} distinct balanced reactions for {size}")

    for kd in kinds:                     # association / dissociation for pressure-dependent
        r = drawer.draw(2, 1)
        reactions.append((r[0], r[1], kd) if r is not None else (*draw_any(), kd))
    covered = set()
    for a, b, _ in reactions:
        covered |= set(a) | set(b)
    inert = {k for k in range(ns) if (comp[k] > 0).sum() == 1 and elements[int(np.argmax(comp[k]))] == "Ar"}
    order = rng.permutation(ns)
    for k in order:                      # every non-inert species takes part in some reaction
        if len(reactions) >= nr:
            break
        if int(k) in covered or int(k) in inert:
            continue
        r = None
        for _ in range(20):
            o1, o2 = types[rng.choice(len(types), p=probs)]
            r = drawer.draw(o1, o2, must_contain=int(k), tries=40)
            if r is not None:
                break
        if r is not None:
            reactions.append((r[0], r[1], KIND_ELEMENTARY))
            covered |= set(r[0]) | set(r[1])
    while len(reactions) < nr:
        r = draw_any()
        reactions.append((r[0], r[1], KIND_ELEMENTARY))
    perm = rng.permutation(nr)
    reactions = [reactions[i] for i in perm]

    nu_f = np.zeros((nr, ns), np.int32)
    nu_r = np.zeros((nr, ns), np.int32)
    kind = np.zeros(nr, np.int32)
    for j, (a, b, kd) in enumerate(reactions):
        dh = sum(n * hf[k] for k, n in b.items()) - sum(n * hf[k] for k, n in a.items())
        if dh > 0:                       # write every reaction in its exothermic direction
            a, b = b, a
        for k, n in a.items():
            nu_f[j, k] = n
        for k, n in b.items():
            nu_r[j, k] = n
        kind[j] = kd

    arrh = np.column_stack([rng.uniform(20.0, 35.0, nr), rng.uniform(-2.0, 2.0, nr),
                            rng.uniform(0.0, 25000.0, nr)])
    eff = np.ones((nr, ns))
    arrh_low = np.zeros((nr, 3))
    troe = np.zeros((nr, 4))
    for j in range(nr):
        if kind[j] == KIND_ELEMENTARY:
            continue
        m = int(rng.integers(3, 7))
        sub = rng.choice(ns, size=min(m, ns), replace=False)
        eff[j, sub] = rng.uniform(0.5, 5.0, len(sub))
        if kind[j] in (KIND_LINDEMANN, KIND_TROE):
            arrh_low[j] = (arrh[j, 0] + rng.uniform(3.0, 8.0), rng.uniform(-2.0, 2.0),
                           rng.uniform(0.0, 0.5) * arrh[j, 2])
        if kind[j] == KIND_TROE:
            t2 = np.exp(rng.uniform(np.log(1000.0), np.log(10000.0))) if rng.random() < 0.5 else 0.0
            troe[j] = (rng.uniform(0.1, 0.9), np.exp(rng.uniform(np.log(10.0), np.log(1000.0))),
                       np.exp(rng.uniform(np.log(500.0), np.log(5000.0))), t2)
    reversible = np.ones(nr, np.int32)
    if n_irreversible:
        reversible[rng.choice(nr, size=n_irreversible, replace=False)] = 0
    return Mechanism(name=size, elements=list(elements), species=names, elem_comp=comp,
                     mol_weight=W, nu_f=nu_f, nu_r=nu_r, arrh=arrh, kind=kind,
                     reversible=reversible, eff=eff, arrh_low=arrh_low, troe=troe, nasa7=nasa,
                     t_mid=t_mid, p_ref=P_BAR, seed=seed,
                     meta={"hf298_over_R": [float(x) for x in hf]})


# ---------------------------------------------------------------------------
# cell states
# ---------------------------------------------------------------------------

def _mass_from_moles(mech, x):
    y = np.asarray(x, float) * mech.mol_weight
    return y / y.sum(-1, keepdims=True)


def _pure(mech, name):
    y = np.zeros(mech.n_species)
    y[mech.species_index(name)] = 1.0
    return y


def _air(mech):
    x = np.zeros(mech.n_species)
    x[mech.species_index("O2")] = 0.21
    if "Ar" in mech.species:
        x[mech.species_index("N2")] = 0.78
        x[mech.species_index("Ar")] = 0.01
    else:
        x[mech.species_index("N2")] = 0.79
    return _mass_from_moles(mech, x)


def _products(mech):
    x = np.zeros(mech.n_species)
    x[mech.species_index("H2O")] = 0.18
    x[mech.species_index("N2")] = 0.72
    if "CO2" in mech.species:
        x[mech.species_index("CO2")] = 0.10
    else:
        x[mech.species_index("N2")] += 0.10
    return _mass_from_moles(mech, x)


def fuel_name(mech) -> str:
    for nm in ("C7H16", "CH4", "H2"):
        if nm in mech.species:
            return nm
    raise ValueError("mechanism has no fuel anchor")


def make_states(mech: Mechanism, n: int, seed: int = 1234, kind: str = "mixture",
                T_range=(800.0, 2800.0), P_atm=(1.0, 50.0)):
    """Seeded batch of cell states (T [K], P [dyn/cm^2], Y [n, ns] mass fractions).

    kind="dirichlet": Y ~ Dirichlet(0.5) over all species, P fixed at P_atm[0].
    kind="mixture":   Y = w_f Y_fuel + w_o Y_air + w_p Y_products, w ~ Dirichlet(1,1,1),
                      plus trace mass fractions logU[1e-12, 1e-4] on every other species;
                      P ~ logU[P_atm].
    """
    rng = np.random.default_rng(np.random.PCG64(seed))
    ns = mech.n_species
    T = rng.uniform(T_range[0], T_range[1], n)
    if kind == "dirichlet":
        P = np.full(n, P_atm[0] * P_ATM)
        Y = rng.dirichlet(np.full(ns, 0.5), size=n)
        Y = np.maximum(Y, 0.0)
        Y /= Y.sum(1, keepdims=True)
        return T, P, Y
    lp = rng.uniform(np.log(P_atm[0]), np.log(P_atm[1]), n)
    P = np.exp(lp) * P_ATM
    w = rng.dirichlet(np.ones(3), size=n)
    base = np.stack([_pure(mech, fuel_name(mech)), _air(mech), _products(mech)])
    Y = w @ base
    trace = np.exp(rng.uniform(np.log(1e-12), np.log(1e-4), (n, ns)))
    Y = np.where(base.sum(0)[None, :] > 0, Y, trace)
    Y /= Y.sum(1, keepdims=True)
    return T, P, Y


def make_ignition_states(mech: Mechanism, n: int, seed: int = 1234,
                         T_range=(900.0, 1400.0), P_atm=(1.0, 20.0), phi_range=(0.5, 2.0)):
    """Fuel / O2 / N2 reactors (N2:O2 = 3.76 molar) at equivalence ratio phi."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    T = rng.uniform(*T_range, n)
    P = rng.uniform(*P_atm, n) * P_ATM
    phi = rng.uniform(*phi_range, n)
    f = mech.species_index(fuel_name(mech))
    comp = dict(zip(mech.elements, mech.elem_comp[f]))
    o2_st = comp.get("C", 0) + comp.get("H", 0) / 4.0 - comp.get("O", 0) / 2.0
    x = np.zeros((n, mech.n_species))
    x[:, f] = phi
    x[:, mech.species_index("O2")] = o2_st
    x[:, mech.species_index("N2")] = 3.76 * o2_st
    return T, P, _mass_from_moles(mech, x), phi


def make_znd_states(mech: Mechanism, n: int, seed: int = 42, s=None):
    """Detonation-channel-like states along s in [0, 1]: T 300 -> 3000 K, P 1 -> 30 atm,
    Y from unburnt fuel/air to products, with trace radicals."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    if s is None:
        s = rng.uniform(0.0, 1.0, n)
    s = np.asarray(s, float)
    T = 300.0 + 2700.0 * s
    P = (1.0 + 29.0 * s) * P_ATM
    fuel = _pure(mech, fuel_name(mech))
    unburnt = 0.06 * fuel + 0.94 * _air(mech)
    Y = (1.0 - s)[:, None] * unburnt[None, :] + s[:, None] * _products(mech)[None, :]
    trace = np.exp(rng.uniform(np.log(1e-12), np.log(1e-5), (n, mech.n_species)))
    Y = Y + trace * (Y == 0)
    Y /= Y.sum(1, keepdims=True)
    return T, P, Y


def subset_indices(n_total: int, n_subset: int, seed: int = 1234) -> np.ndarray:
    """Fixed parity subset: the first ``n_subset`` cells of a seeded permutation."""
    rng = np.random.default_rng(np.random.PCG64(seed + 7))
    return np.sort(rng.permutation(n_total)[:n_subset])
