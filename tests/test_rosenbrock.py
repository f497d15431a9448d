"""The integrator's Rosenbrock coefficients (read from the library, no GPU needed) against
the order conditions and stability properties that define the method (Hairer & Wanner,
Solving ODEs II, Sec. IV.7, Table 7.1; Rodas3 of Sandu et al. 1997: order 3, embedded
order 2, stiffly accurate, L-stable)."""
import numpy as np
import pytest

from paper_2008_08483_gb300 import build as B
from paper_2008_08483_gb300 import chem


@pytest.fixture(scope="module")
def tab():
    B.build()
    return chem.rosenbrock_tableau()


def _parts(t):
    a, g, gii = t["alpha"], t["gamma"], t["gamma_ii"]
    beta = a + g                      # strictly lower beta_ij = alpha_ij + gamma_ij
    bp = beta.sum(1)                  # beta'_i
    al = a.sum(1)                     # alpha_i
    return a, g, gii, beta, bp, al


def test_shape(tab):
    assert tab["stages"] == 4
    assert np.all(np.triu(tab["alpha"]) == 0) and np.all(np.triu(tab["gamma"]) == 0)


def test_order_conditions(tab):
    a, g, gii, beta, bp, al = _parts(tab)
    b, bh = tab["b"], tab["bhat"]
    # order 1 and 2
    assert np.isclose(b.sum(), 1.0, atol=1e-15)
    assert np.isclose(b @ bp, 0.5 - gii, atol=1e-15)
    # order 3
    assert np.isclose(b @ al ** 2, 1.0 / 3.0, atol=1e-15)
    assert np.isclose(b @ (beta @ bp), 1.0 / 6.0 - gii + gii ** 2, atol=1e-15)
    # embedded solution: order 2
    assert np.isclose(bh.sum(), 1.0, atol=1e-15)
    assert np.isclose(bh @ bp, 0.5 - gii, atol=1e-15)
    # and not order 3, so that b - bhat estimates the local error
    assert not np.isclose(bh @ al ** 2, 1.0 / 3.0) or \
        not np.isclose(bh @ (beta @ bp), 1.0 / 6.0 - gii + gii ** 2)


def test_stiffly_accurate(tab):
    a, g, gii, beta, bp, al = _parts(tab)
    s = tab["stages"]
    assert np.allclose(tab["b"][:s - 1], beta[s - 1, :s - 1], atol=1e-15)
    assert np.isclose(tab["b"][s - 1], gii)
    assert np.allclose(tab["bhat"][:s - 2], beta[s - 2, :s - 2], atol=1e-15)
    assert np.isclose(tab["bhat"][s - 2], gii)


def _R(tab, z, b):
    s = tab["stages"]
    full = tab["alpha"] + tab["gamma"] + tab["gamma_ii"] * np.eye(s)
    return 1.0 + z * b @ np.linalg.solve(np.eye(s) - z * full, np.ones(s))


def test_stability_function(tab):
    # R(z) - e^z = O(z^4) (order 3), L-stable: |R(iy)| <= 1 and R(-inf) = 0
    e1 = abs(_R(tab, 0.02, tab["b"]) - np.exp(0.02))
    e2 = abs(_R(tab, 0.01, tab["b"]) - np.exp(0.01))
    assert 3.7 < np.log2(e1 / e2) < 4.3
    assert max(abs(_R(tab, 1j * y, tab["b"])) for y in np.logspace(-3, 6, 300)) <= 1.0 + 1e-12
    assert abs(_R(tab, -1e12, tab["b"])) < 1e-9
    rng = np.random.default_rng(0)
    z = -rng.uniform(0, 1e3, 500) + 1j * rng.uniform(-1e3, 1e3, 500)
    assert max(abs(_R(tab, zz, tab["b"])) for zz in z) <= 1.0 + 1e-12
