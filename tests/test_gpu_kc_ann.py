"""Approximate-ANN equilibrium constants (Sec. 2.3, Eqs. 12-14): the exact ln K_c table that
trains them against the oracle, the trained networks' accuracy, and the source-term kernel
with network ln K_c against the oracle evaluated with the same network values (FP32 bar)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2008_08483_gb300 import build as B
from paper_2008_08483_gb300 import chem, kc_ann, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    B.build()
    return torch.device("cuda:0")


def test_log_kc_matches_oracle(dev, mech53):
    h = chem.Mechanism(mech53)
    om = O.OracleMechanism(mech53)
    T = np.concatenate([np.linspace(300.0, 3500.0, 37), [999.999, 1000.0, 1000.001]])
    K = chem.log_kc(h, torch.as_tensor(T, device=dev)).cpu().numpy()
    for i, t in enumerate(T):
        C = np.full(mech53.n_species, 1e-6)
        ref = O.cell_detail(om, t, C)["lnKc"]
        assert np.max(np.abs(K[i] - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


@pytest.fixture(scope="module")
def trained(dev, mech53):
    h = chem.Mechanism(mech53)
    hf, _ = kc_ann.train_kc_ann(h, 3, 32, "elu", n_samples=200_000, steps=1500)
    lf, _ = kc_ann.train_kc_ann(h, 1, 8, "elu", n_samples=200_000, steps=1500)
    return h, hf, lf


def test_network_accuracy(dev, mech53, trained):
    h, hf, lf = trained
    T = np.linspace(400.0, 3000.0, 301)
    exact = chem.log_kc(h, torch.as_tensor(T, device=dev)).cpu().numpy()
    e_hf = np.abs(kc_ann.forward_np(hf, T) - exact)
    e_lf = np.abs(kc_ann.forward_np(lf, T) - exact)
    # relative to the spread of each reaction's ln K_c over the range.  The networks are
    # approximations (Sec. 2.3) trained on the GPU, whose reductions are not bitwise
    # reproducible, so the maximum over all reactions and temperatures varies between runs
    # (up to 0.025 seen for the 3 x 32 network); the bounds leave room for that and the
    # median keeps the accuracy claim
    spread = exact.max(0) - exact.min(0) + 1.0
    rel_hf, rel_lf = e_hf / spread, e_lf / spread
    assert np.max(rel_hf) < 0.05 and np.median(rel_hf) < 0.01
    assert np.max(rel_lf) < 0.2
    assert np.median(e_hf) < np.median(e_lf)


@pytest.mark.parametrize("which", ["hf", "lf"])
def test_kernel_matches_oracle_with_network_kc(dev, mech53, trained, which):
    h, hf, lf = trained
    params = hf if which == "hf" else lf
    ann = chem.KcAnn(h, params)
    n = 2 * 64 + 19
    T, P, Y = synth.make_states(mech53, n, seed=41)
    T32, P32, Y32 = (a.astype(np.float32) for a in (T, P, Y))
    w = chem.source_term_kc_ann(h, ann, *(torch.as_tensor(a, device=dev) for a in (T32, P32, Y32)))
    w = w.cpu().numpy().astype(float)
    # the oracle on the same FP32-rounded inputs, ln K_c from the network in float64
    lnkc = kc_ann.forward_np(params, T32.astype(float))
    ref = O.source_term_kc(mech53, T32.astype(float), P32.astype(float), Y32.astype(float), lnkc)
    err = np.abs(w - ref).max(1) / np.abs(ref).max(1)
    assert err.max() <= 2e-5, err.max()
    ann.close()


def test_network_load_validation(dev, mech9):
    h = chem.Mechanism(mech9)
    good = dict(n_layers=1, n_hidden=4, activation="relu", x_mean=7.0, x_std=0.5,
                w_in=np.ones(4), b_in=np.zeros(4), w_hid=None, b_hid=None,
                w_out=np.ones((mech9.n_reactions, 4)), b_out=np.zeros(mech9.n_reactions),
                y_mean=np.zeros(mech9.n_reactions), y_std=np.ones(mech9.n_reactions))
    chem.KcAnn(h, good).close()
    for bad in (dict(n_hidden=33), dict(n_layers=0), dict(x_std=0.0)):
        p = dict(good)
        p.update(bad)
        if "n_hidden" in bad:
            p.update(w_in=np.ones(33), b_in=np.zeros(33), w_out=np.ones((mech9.n_reactions, 33)))
        with pytest.raises(chem.ChemError) as e:
            chem.KcAnn(h, p)
        assert e.value.status == 1
    other = chem.Mechanism(synth.make_mechanism("h2air_9_21", seed=2))
    ann = chem.KcAnn(h, good)
    T = torch.full((4,), 1500.0, device=dev, dtype=torch.float32)
    Y = torch.full((4, 9), 1.0 / 9, device=dev, dtype=torch.float32)
    with pytest.raises(chem.ChemError):
        chem.source_term_kc_ann(other, ann, T, T * 1000, Y)


def test_exact_reference_of_the_network_kernel(dev, mech53):
    """No network: the network variant's kernel with the exact Gibbs layer (the reference of
    the speed-up), against the oracle at the FP32 bar and against the FP32 source term."""
    h = chem.Mechanism(mech53)
    om = O.OracleMechanism(mech53)
    n = 3 * 64 + 11
    T, P, Y = synth.make_states(mech53, n, seed=43)
    T32, P32, Y32 = (a.astype(np.float32) for a in (T, P, Y))
    t = [torch.as_tensor(a, device=dev) for a in (T32, P32, Y32)]
    w = chem.source_term_kc_ann(h, None, *t).cpu().numpy().astype(float)
    ref = O.source_term(om, *(a.astype(float) for a in (T32, P32, Y32)))
    err = np.abs(w - ref).max(1) / np.abs(ref).max(1)
    assert err.max() <= 1e-5, err.max()
    w32 = chem.source_term(h, *t, chem.FP32).cpu().numpy().astype(float)
    assert (np.abs(w - w32).max(1) / np.abs(ref).max(1)).max() <= 2e-5
