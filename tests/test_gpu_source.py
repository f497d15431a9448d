"""Parity of the CUDA source-term paths with the FP64 CPU oracle, element by element,
through the C ABI.

Error measure: per cell, max_k |omega_gpu - omega_oracle| / max_k |omega_oracle|.
Bars: 1e-10 for FP64, 1e-5 for FP32, 1e-4 for split BF16.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2008_08483_gb300 import build as B
from paper_2008_08483_gb300 import chem, synth

pytestmark = pytest.mark.gpu

TOL = {chem.FP64: 1e-10, chem.FP32: 1e-5, chem.SPLIT_BF16: 1e-4}
STATES = {  # (state kind, T range, P range in atm) of each workload
    "h2air_9_21": ("dirichlet", (1000.0, 2500.0), (1.0, 1.0)),
    "gri_53_325": ("mixture", (800.0, 2800.0), (1.0, 50.0)),
    "heavy_160_1000": ("mixture", (700.0, 2600.0), (1.0, 100.0)),
}


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    B.build()
    return torch.device("cuda:0")


_mechs = {}


def loaded(size, seed=1, **kw):
    key = (size, seed, tuple(sorted(kw.items())))
    if key not in _mechs:
        m = synth.make_mechanism(size, seed=seed, **kw)
        _mechs[key] = (m, chem.Mechanism(m), O.OracleMechanism(m))
    return _mechs[key]


def states(m, size, n, seed=1234):
    kind, Tr, Pr = STATES[size]
    return synth.make_states(m, n, seed=seed, kind=kind, T_range=Tr, P_atm=Pr)


def run(h, T, P, Y, prec, dev, ldY=None, ldO=None):
    dt = torch.float64 if prec == chem.FP64 else torch.float32
    n, ns = Y.shape
    ldY = ldY or ns
    ldO = ldO or ns
    Yb = torch.zeros((n, ldY), dtype=dt, device=dev)
    Yb[:, :ns] = torch.as_tensor(Y, dtype=dt)
    ob = torch.full((n, ldO), 12345.0, dtype=dt, device=dev)
    chem.source_term(h, torch.as_tensor(T, dtype=dt, device=dev),
                     torch.as_tensor(P, dtype=dt, device=dev), Yb[:, :ns], prec,
                     out=ob[:, :ns])
    torch.cuda.synchronize()
    if prec == chem.SPLIT_BF16:
        assert h.device_status() == 0, "a tensor-core kernel gave up on a bounded wait"
    o = ob.cpu().numpy().astype(np.float64)
    return o[:, :ns], o[:, ns:]


def cell_err(w, ref):
    return np.abs(w - ref).max(1) / np.abs(ref).max(1)


def as_prec(x, prec):
    """The inputs as the path sees them (FP32 paths read float copies)."""
    return np.asarray(x, np.float32).astype(np.float64) if prec != chem.FP64 else x


PATHS = [chem.FP64, chem.FP32, chem.SPLIT_BF16]
# the split-precision path: tables resident in shared memory up to 53 species (64 contraction-1
# columns: species, log2 c_tot, the normalisation and nine Arrhenius rows), streamed beyond,
# up to 192 species (omega columns in tensor memory)
BF16_MAX_SPECIES = 192


@pytest.mark.parametrize("prec", PATHS)
@pytest.mark.parametrize("size,n", [("h2air_9_21", 1024), ("gri_53_325", 5 * 64 + 37),
                                    ("heavy_160_1000", 3 * 32 + 5)])
def test_parity_with_oracle(dev, prec, size, n):
    m, h, om = loaded(size)
    T, P, Y = states(m, size, n, seed=77)
    T, P, Y = as_prec(T, prec), as_prec(P, prec), as_prec(Y, prec)
    if prec == chem.SPLIT_BF16 and m.n_species > BF16_MAX_SPECIES:
        with pytest.raises(chem.ChemError) as e:
            run(h, T, P, Y, prec, dev)
        assert e.value.status == 4            # CHEM_EUNSUPPORTED, nothing launched
        return
    ref = O.source_term(om, T, P, Y)
    w, _ = run(h, T, P, Y, prec, dev)
    err = cell_err(w, ref)
    assert err.max() <= TOL[prec], f"worst cell {err.argmax()} err {err.max():.3e}"


@pytest.mark.parametrize("prec", PATHS)
def test_all_reaction_kinds(dev, prec):
    """Lindemann, Troe, third-body and irreversible reactions together."""
    m, h, om = loaded("gri_53_325", seed=5, n_lindemann=6, n_irreversible=25)
    assert set(np.unique(m.kind)) == {0, 1, 2, 3} and (m.reversible == 0).sum() == 25
    T, P, Y = states(m, "gri_53_325", 300, seed=3)
    T, P, Y = as_prec(T, prec), as_prec(P, prec), as_prec(Y, prec)
    ref = O.source_term(om, T, P, Y)
    w, _ = run(h, T, P, Y, prec, dev)
    assert cell_err(w, ref).max() <= TOL[prec]


@pytest.mark.parametrize("prec", PATHS)
def test_conservation_of_gpu_output(dev, prec):
    m, h, om = loaded("gri_53_325")
    T, P, Y = states(m, "gri_53_325", 500, seed=4)
    w, _ = run(h, T, P, Y, prec, dev)
    mass = np.abs(w @ m.mol_weight) / (np.abs(w) @ m.mol_weight)
    E = m.elem_comp.astype(float)
    el = np.abs(w @ E) / np.maximum(np.abs(w) @ E, 1e-300)
    bar = 1e-12 if prec == chem.FP64 else 1e-6
    assert mass.max() < bar and el.max() < bar


@pytest.mark.parametrize("prec", PATHS)
def test_edge_cases(dev, prec):
    m, h, om = loaded("h2air_9_21")
    ns = m.n_species
    T, P, Y = states(m, "h2air_9_21", 70, seed=9)
    Y = Y.copy()
    Y[3, 2] = 0.0                      # an absent species
    Y[5, 4] = -1e-3                    # a negative mass fraction counts as zero
    Y[7, :] = 0.0                      # an all-zero row: every concentration is zero
    T, P, Y = as_prec(T, prec), as_prec(P, prec), as_prec(Y, prec)
    ref = O.source_term(om, T, P, Y)
    # padded leading dimensions; the padding columns of omega are not written
    w, pad = run(h, T, P, Y, prec, dev, ldY=ns + 3, ldO=ns + 5)
    assert np.all(pad == 12345.0)
    live = np.ones(len(T), bool)
    live[7] = False
    assert cell_err(w[live], ref[live]).max() <= TOL[prec]
    assert np.all(ref[7] == 0.0) and np.all(np.abs(w[7]) < 1e-30)
    # zero cells: a no-op
    dt = torch.float64 if prec == chem.FP64 else torch.float32
    e = torch.empty((0,), dtype=dt, device=dev)
    chem.source_term(h, e, e, torch.empty((0, ns), dtype=dt, device=dev), prec)


def test_argument_errors(dev):
    m, h, om = loaded("h2air_9_21")
    T = torch.ones(4, dtype=torch.float64, device=dev)
    Y = torch.ones((4, m.n_species), dtype=torch.float64, device=dev)
    L = chem.lib()
    import ctypes as C
    rc = L.chem_source_term(h.handle, 4, T.data_ptr(), T.data_ptr(), Y.data_ptr(),
                            m.n_species - 1, Y.data_ptr(), m.n_species, 0, None)
    assert rc == 1 and b"ldY" in L.chem_last_error()
    rc = L.chem_source_term(h.handle, -1, T.data_ptr(), T.data_ptr(), Y.data_ptr(),
                            m.n_species, Y.data_ptr(), m.n_species, 0, None)
    assert rc == 1
    rc = L.chem_source_term(h.handle, 4, T.data_ptr(), T.data_ptr(), Y.data_ptr(),
                            m.n_species, Y.data_ptr(), m.n_species, 9, None)
    assert rc == 1


@pytest.mark.parametrize("prec", PATHS)
def test_full_size_sampled(dev, prec):
    """53 species / 325 reactions at 2^20 cells, the benchmark's launch: sampled cells
    against the oracle."""
    m, h, om = loaded("gri_53_325")
    n = 1 << 20
    T, P, Y = states(m, "gri_53_325", n, seed=1234)
    T, P, Y = as_prec(T, prec), as_prec(P, prec), as_prec(Y, prec)
    w, _ = run(h, T, P, Y, prec, dev)
    idx = synth.subset_indices(n, 4096)
    idx = np.concatenate([idx, [0, n - 1]])
    ref = O.source_term(om, T[idx], P[idx], Y[idx])
    assert cell_err(w[idx], ref).max() <= TOL[prec]


@pytest.mark.parametrize("prec", [chem.SPLIT_BF16, chem.FP32])
def test_full_size_sampled_160_1000(dev, prec):
    """160 species / 1000 reactions at 2^18 cells (the large-mechanism workload's launch) on
    the split-precision and FP32 paths: sampled cells and the last cell against the oracle."""
    m, h, om = loaded("heavy_160_1000")
    n = 1 << 18
    T, P, Y = states(m, "heavy_160_1000", n, seed=1234)
    T, P, Y = (as_prec(x, prec) for x in (T, P, Y))
    w, _ = run(h, T, P, Y, prec, dev)
    idx = np.concatenate([synth.subset_indices(n, 1024), [0, n - 1]])
    ref = O.source_term(om, T[idx], P[idx], Y[idx])
    assert cell_err(w[idx], ref).max() <= TOL[prec]


def with_inert_species(m, extra):
    """The mechanism with `extra` species appended that take part in no reaction (copies of
    the first species' thermodynamics and composition, default third-body efficiency)."""
    import dataclasses
    ns, nr = m.n_species, m.n_reactions
    pad = lambda a, v: np.concatenate([a, np.full((nr, extra), v, a.dtype)], axis=1)
    return dataclasses.replace(
        m, name=f"{m.name}+{extra}inert", species=m.species + [f"INERT{i}" for i in range(extra)],
        elem_comp=np.concatenate([m.elem_comp, np.repeat(m.elem_comp[:1], extra, 0)]),
        mol_weight=np.concatenate([m.mol_weight, np.repeat(m.mol_weight[:1], extra)]),
        nu_f=pad(m.nu_f, 0), nu_r=pad(m.nu_r, 0), eff=pad(m.eff, 1.0),
        nasa7=np.concatenate([m.nasa7, np.repeat(m.nasa7[:1], extra, 0)]))


@pytest.mark.parametrize("size,extra", [("h2air_9_21", 14), ("gri_53_325", 5)])
def test_bf16_species_padding(dev, size, extra):
    """Species counts between the padded column widths: 23 species (34 of 64 contraction-1
    columns, tables resident in shared memory) and 58 species (69 columns, past the resident
    tables: the streamed-table kernel), both against the oracle."""
    base, _, _ = loaded(size)
    m = with_inert_species(base, extra)
    h, om = chem.Mechanism(m), O.OracleMechanism(m)
    T, P, Yb = states(base, size, 3 * 128 + 19, seed=21)
    rng = np.random.default_rng(5)
    Y = np.concatenate([Yb, rng.uniform(0.0, 0.02, (len(T), extra))], axis=1)
    Y /= Y.sum(axis=1, keepdims=True)
    T, P, Y = (as_prec(x, chem.SPLIT_BF16) for x in (T, P, Y))
    if m.n_species > BF16_MAX_SPECIES:
        with pytest.raises(chem.ChemError) as e:
            run(h, T, P, Y, chem.SPLIT_BF16, dev)
        assert e.value.status == 4
        return
    ref = O.source_term(om, T, P, Y)
    w, _ = run(h, T, P, Y, chem.SPLIT_BF16, dev)
    assert np.all(w[:, base.n_species:] == 0.0)
    assert cell_err(w, ref).max() <= TOL[chem.SPLIT_BF16]


@pytest.mark.parametrize("n", [3 * 4864 + 17, 70001])
def test_fp32_intermediate_cells_per_warp(dev, n):
    """Batch sizes for which the FP32 kernel's blocks are neither one warp nor the widest
    (here 4 and 6 warps of 32 cells, with a ragged last warp): sampled cells and the tail
    against the oracle."""
    m, h, om = loaded("gri_53_325")
    T, P, Y = states(m, "gri_53_325", n, seed=31)
    T, P, Y = (as_prec(x, chem.FP32) for x in (T, P, Y))
    w, _ = run(h, T, P, Y, chem.FP32, dev)
    idx = np.concatenate([synth.subset_indices(n, 512), np.arange(n - 40, n)])
    ref = O.source_term(om, T[idx], P[idx], Y[idx])
    assert cell_err(w[idx], ref).max() <= TOL[chem.FP32]


def test_fp32_extreme_states(dev):
    """FP32 at the edges of its arithmetic: T at the NASA-7 range switch (t_mid and the
    floats either side of it) and at 300 K and 3500 K, pressures from 0.01 to 100 atm, and
    mass fractions down to the FP32 subnormal range (1e-40) next to ordinary ones."""
    m, h, om = loaded("gri_53_325")
    ns = m.n_species
    T0, P0, Y0 = states(m, "gri_53_325", 96, seed=77)
    tm = np.float32(m.t_mid)
    Ts = np.array([300.0, 3500.0, tm, np.nextafter(tm, np.float32(0)),
                   np.nextafter(tm, np.float32(1e9))], np.float64)
    T = Ts[np.arange(96) % len(Ts)]
    P = np.where(np.arange(96) % 2 == 0, 0.01, 100.0) * 1.01325e6
    Y = Y0.copy()
    Y[1::3, 5] = 1e-40                 # subnormal in FP32
    Y[2::3, 7] = 1e-30
    Y[::5, 9] = 3e-39
    T, P, Y = (as_prec(x, chem.FP32) for x in (T, P, Y))
    ref = O.source_term(om, T, P, Y)
    w, _ = run(h, T, P, Y, chem.FP32, dev)
    assert np.all(np.isfinite(w))
    assert cell_err(w, ref).max() <= TOL[chem.FP32]


def test_fp32_warp_kernel_fallback(dev):
    """A mechanism the thread-per-cell FP32 kernel does not take (a reaction with four
    reactant species: a spectator added to both sides of a three-reactant reaction, which
    keeps element balance and the net stoichiometry) runs the warp-per-cell kernel, at the
    same bar against the oracle."""
    import dataclasses
    base, _, _ = loaded("gri_53_325")
    nf = (base.nu_f > 0).sum(1)
    j = int(np.nonzero(nf == 3)[0][0])
    k = int(np.nonzero((base.nu_f[j] == 0) & (base.nu_r[j] == 0))[0][0])
    nu_f, nu_r = base.nu_f.copy(), base.nu_r.copy()
    nu_f[j, k] += 1
    nu_r[j, k] += 1
    m = dataclasses.replace(base, name=base.name + "+spectator", nu_f=nu_f, nu_r=nu_r)
    h, om = chem.Mechanism(m), O.OracleMechanism(m)
    T, P, Y = states(m, "gri_53_325", 2 * 32 + 9, seed=5)
    T, P, Y = (as_prec(x, chem.FP32) for x in (T, P, Y))
    ref = O.source_term(om, T, P, Y)
    w, _ = run(h, T, P, Y, chem.FP32, dev)
    assert cell_err(w, ref).max() <= TOL[chem.FP32]
