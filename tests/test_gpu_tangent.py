"""jvp / vjp / dense Jacobian kernels of omega(T, ln C) against the oracle's analytic
Jacobian (itself pinned to central differences), the adjoint identity, and the autograd
path.  Bars: 1e-10 (FP64) and 2e-5 (FP32) per cell, relative to the cell's largest entry."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2008_08483_gb300 import build as B
from paper_2008_08483_gb300 import chem, synth

pytestmark = pytest.mark.gpu
TOL = {chem.FP64: 1e-10, chem.FP32: 2e-5}


@pytest.fixture(scope="module")
def setup():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    B.build()
    dev = torch.device("cuda:0")
    m = synth.make_mechanism("gri_53_325", seed=3, n_lindemann=4, n_irreversible=8)
    h = chem.Mechanism(m)
    om = O.OracleMechanism(m)
    n = 3 * 64 + 11
    T, P, Y = synth.make_states(m, n, seed=31, T_range=(700.0, 2700.0))
    C = np.stack([O.concentrations(om, T[i], P[i], Y[i]) for i in range(n)])
    J = np.zeros((n, m.n_species, m.n_species + 1))
    for i in range(n):
        Jc, dT = O.jacobian_tc(om, T[i], C[i])
        J[i, :, :-1], J[i, :, -1] = Jc, dT
    return dict(dev=dev, m=m, h=h, om=om, T=T, lnC=np.log(C), J=J)


def tens(x, prec, dev):
    return torch.as_tensor(x, dtype=torch.float64 if prec == chem.FP64 else torch.float32,
                           device=dev)


def cellrel(a, b):
    a, b = np.asarray(a, float).reshape(len(a), -1), np.asarray(b, float).reshape(len(b), -1)
    return (np.abs(a - b).max(1) / np.abs(b).max(1)).max()


@pytest.mark.parametrize("prec", [chem.FP64, chem.FP32])
def test_jacobian_entry(setup, prec):
    s = setup
    J = chem.source_term_jacobian(s["h"], tens(s["T"], prec, s["dev"]),
                                  tens(s["lnC"], prec, s["dev"]), prec)
    torch.cuda.synchronize()
    assert cellrel(J.double().cpu().numpy(), s["J"]) <= TOL[prec]


@pytest.mark.parametrize("prec", [chem.FP64, chem.FP32])
def test_jvp_and_omega(setup, prec):
    s = setup
    rng = np.random.default_rng(5)
    dT = rng.normal(size=len(s["T"])) * 10.0
    dl = rng.normal(size=s["lnC"].shape)
    om, dom = chem.source_term_jvp(s["h"], tens(s["T"], prec, s["dev"]),
                                   tens(s["lnC"], prec, s["dev"]), tens(dT, prec, s["dev"]),
                                   tens(dl, prec, s["dev"]), prec)
    torch.cuda.synchronize()
    expect = np.einsum("ikm,im->ik", s["J"][:, :, :-1], dl) + s["J"][:, :, -1] * dT[:, None]
    assert cellrel(dom.double().cpu().numpy(), expect) <= TOL[prec]
    ref = O.source_term_tc(s["om"], s["T"], np.exp(s["lnC"]))
    assert cellrel(om.double().cpu().numpy(), ref) <= TOL[prec]


@pytest.mark.parametrize("prec", [chem.FP64, chem.FP32])
def test_vjp(setup, prec):
    s = setup
    g = np.random.default_rng(6).normal(size=s["lnC"].shape)
    gT, glnC = chem.source_term_vjp(s["h"], tens(s["T"], prec, s["dev"]),
                                    tens(s["lnC"], prec, s["dev"]), tens(g, prec, s["dev"]), prec)
    torch.cuda.synchronize()
    eT = np.einsum("ik,ik->i", s["J"][:, :, -1], g)
    eC = np.einsum("ikm,ik->im", s["J"][:, :, :-1], g)
    both = np.concatenate([glnC.double().cpu().numpy(), gT.double().cpu().numpy()[:, None]], 1)
    assert cellrel(both, np.concatenate([eC, eT[:, None]], 1)) <= TOL[prec]


@pytest.mark.parametrize("prec", [chem.FP64, chem.FP32])
def test_jvp_vjp_large_mechanism(setup, prec):
    """jvp and vjp at 160 species / 1000 reactions (90 third-body, 75 Troe) against the
    oracle's analytic Jacobian, and a batch (2 * 64 + 5 cells) that ends in a partial block."""
    dev = setup["dev"]
    m = synth.make_mechanism("heavy_160_1000", seed=1)
    h, om = chem.Mechanism(m), O.OracleMechanism(m)
    n = 2 * 64 + 5
    T, P, Y = synth.make_states(m, n, seed=41, T_range=(700.0, 2600.0))
    C = np.stack([O.concentrations(om, T[i], P[i], Y[i]) for i in range(n)])
    J = np.zeros((n, m.n_species, m.n_species + 1))
    for i in range(n):
        Jc, dTc = O.jacobian_tc(om, T[i], C[i])
        J[i, :, :-1], J[i, :, -1] = Jc, dTc
    rng = np.random.default_rng(8)
    dT, dl, g = rng.normal(size=n) * 10.0, rng.normal(size=C.shape), rng.normal(size=C.shape)
    Tt, lt = tens(T, prec, dev), tens(np.log(C), prec, dev)
    _, dom = chem.source_term_jvp(h, Tt, lt, tens(dT, prec, dev), tens(dl, prec, dev), prec)
    gT, gl = chem.source_term_vjp(h, Tt, lt, tens(g, prec, dev), prec)
    torch.cuda.synchronize()
    expect = np.einsum("ikm,im->ik", J[:, :, :-1], dl) + J[:, :, -1] * dT[:, None]
    assert cellrel(dom.double().cpu().numpy(), expect) <= TOL[prec]
    eT = np.einsum("ik,ik->i", J[:, :, -1], g)
    eC = np.einsum("ikm,ik->im", J[:, :, :-1], g)
    both = np.concatenate([gl.double().cpu().numpy(), gT.double().cpu().numpy()[:, None]], 1)
    assert cellrel(both, np.concatenate([eC, eT[:, None]], 1)) <= TOL[prec]
    h.close()


def test_adjoint_identity(setup):
    """<g, J v> = <J^T g, v> between the two kernels, per cell."""
    s = setup
    prec, dev = chem.FP64, s["dev"]
    rng = np.random.default_rng(7)
    v_T, v_l = rng.normal(size=len(s["T"])), rng.normal(size=s["lnC"].shape)
    g = rng.normal(size=s["lnC"].shape)
    T, l = tens(s["T"], prec, dev), tens(s["lnC"], prec, dev)
    _, jv = chem.source_term_jvp(s["h"], T, l, tens(v_T, prec, dev), tens(v_l, prec, dev), prec,
                                 with_omega=False)
    gT, gl = chem.source_term_vjp(s["h"], T, l, tens(g, prec, dev), prec)
    lhs = (jv.cpu().numpy() * g).sum(1)
    rhs = (gl.cpu().numpy() * v_l).sum(1) + gT.cpu().numpy() * v_T
    scale = np.abs(jv.cpu().numpy() * g).sum(1)
    assert np.all(np.abs(lhs - rhs) <= 1e-12 * scale)


def test_autograd_backward_and_finite_differences(setup):
    """torch.autograd through chem.omega (backward = vjp kernel) against central
    differences of the FP64 forward kernel."""
    s = setup
    dev = s["dev"]
    T = tens(s["T"][:16], chem.FP64, dev).requires_grad_(True)
    l = tens(s["lnC"][:16], chem.FP64, dev).requires_grad_(True)
    g = torch.as_tensor(np.random.default_rng(8).normal(size=(16, s["m"].n_species)), device=dev)
    w = chem.omega(s["h"], T, l)
    (w * g).sum().backward()
    with torch.no_grad():
        fd_T = torch.zeros(16, dtype=torch.float64, device=dev)
        for sign in (1.0, -1.0):
            Tp = T + sign * 1e-6 * T
            wp = chem.omega(s["h"], Tp, l)
            fd_T += sign * (wp * g).sum(1) / (2e-6 * T)
    assert torch.allclose(T.grad, fd_T, rtol=1e-6, atol=1e-6 * float(fd_T.abs().max()))
    # directional derivative along a random direction over all of ln C, so that it has
    # the magnitude of the Jacobian (single trace-species derivatives drown in rounding)
    with torch.no_grad():
        v = torch.as_tensor(np.random.default_rng(9).normal(size=tuple(l.shape)), device=dev)
        fd_l = ((chem.omega(s["h"], T, l + 1e-6 * v) - chem.omega(s["h"], T, l - 1e-6 * v)) * g
                ).sum(1) / 2e-6
        an_l = (l.grad * v).sum(1)
    assert torch.allclose(an_l, fd_l, rtol=1e-6, atol=1e-6 * float(fd_l.abs().max()))


def test_split_bf16_is_not_a_derivative_precision(setup):
    s = setup
    with pytest.raises(chem.ChemError) as e:
        chem.source_term_vjp(s["h"], tens(s["T"], chem.FP32, s["dev"]),
                             tens(s["lnC"], chem.FP32, s["dev"]),
                             tens(np.zeros_like(s["lnC"]), chem.FP32, s["dev"]), chem.SPLIT_BF16)
    assert e.value.status == 4
