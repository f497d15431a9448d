"""Training of the approximate-ANN equilibrium constants (Sec. 2.3, Eqs. 12-14; "Arch 2":
the network's only input is ln T).

The training set is a sweep of temperatures with the exact ln K_c of every reaction from the
library (chem_log_kc: the Gibbs layer folded through the net stoichiometry, Eqs. 8-11);
inputs and targets are standardised and the mean squared error is minimised (Sec. 3.1.1).
Training is an offline preparation step done once per mechanism with PyTorch; the trained
weights are then evaluated inside the library's source-term kernel
(chem_source_term_kc_ann).
"""
from __future__ import annotations

import numpy as np

from . import chem


def train_kc_ann(mech: chem.Mechanism, n_layers: int = 3, n_hidden: int = 32,
                 activation: str = "elu", T_range=(250.0, 3500.0), n_samples: int = 1_000_000,
                 steps: int = 3000, batch: int = 16384, lr: float = 3e-3, seed: int = 0,
                 device: str = "cuda"):
    """Train a network ln T -> ln K_c [n_reactions]; returns the parameter dict of KcAnn
    (float32 arrays) and the training history."""
    import torch

    gen = torch.Generator(device="cpu").manual_seed(seed)
    T = torch.empty(n_samples, dtype=torch.float64).uniform_(*T_range, generator=gen)
    Td = T.to(device)
    Y = chem.log_kc(mech, Td)                               # exact targets, FP64
    x = torch.log(Td)
    x_mean, x_std = float(x.mean()), float(x.std())
    y_mean, y_std = Y.mean(0), Y.std(0).clamp_min(1e-6)
    xs = ((x - x_mean) / x_std).float().unsqueeze(1)
    ys = ((Y - y_mean) / y_std).float()
    act = {"relu": torch.nn.ReLU, "elu": torch.nn.ELU}[activation]
    layers = [torch.nn.Linear(1, n_hidden), act()]
    for _ in range(n_layers - 1):
        layers += [torch.nn.Linear(n_hidden, n_hidden), act()]
    layers.append(torch.nn.Linear(n_hidden, mech.n_reactions))
    torch.manual_seed(seed)
    net = torch.nn.Sequential(*layers).to(device)
    opt = torch.optim.Adam(net.parameters(), lr=lr)
    sched = torch.optim.lr_scheduler.CosineAnnealingLR(opt, steps)
    hist = []
    for step in range(steps):
        idx = torch.randint(0, n_samples, (batch,), device=device)
        loss = torch.mean((net(xs[idx]) - ys[idx]) ** 2)
        opt.zero_grad(set_to_none=True)
        loss.backward()
        opt.step()
        sched.step()
        if step % 100 == 0 or step == steps - 1:
            hist.append((step, float(loss.detach())))
    lin = [m for m in net if isinstance(m, torch.nn.Linear)]
    cpu = lambda t: t.detach().float().cpu().numpy()
    params = dict(
        n_layers=n_layers, n_hidden=n_hidden, activation=activation, x_mean=x_mean,
        x_std=x_std, w_in=cpu(lin[0].weight[:, 0]), b_in=cpu(lin[0].bias),
        w_hid=(np.stack([cpu(l.weight) for l in lin[1:-1]]) if n_layers > 1 else None),
        b_hid=(np.stack([cpu(l.bias) for l in lin[1:-1]]) if n_layers > 1 else None),
        w_out=cpu(lin[-1].weight), b_out=cpu(lin[-1].bias), y_mean=cpu(y_mean),
        y_std=cpu(y_std), T_range=tuple(T_range))
    return params, hist


def forward_np(params, T):
    """The network in float64 numpy (ln K_c [len(T), n_reactions]), for checks."""
    a = (np.log(np.asarray(T, float)) - params["x_mean"]) / params["x_std"]
    act = (lambda v: np.maximum(v, 0.0)) if params["activation"] == "relu" else \
        (lambda v: np.where(v > 0, v, np.expm1(np.minimum(v, 0.0))))
    h = act(a[:, None] * params["w_in"][None, :].astype(float) + params["b_in"].astype(float))
    for l in range(params["n_layers"] - 1):
        h = act(h @ params["w_hid"][l].astype(float).T + params["b_hid"][l].astype(float))
    out = h @ params["w_out"].astype(float).T + params["b_out"].astype(float)
    return params["y_mean"].astype(float) + params["y_std"].astype(float) * out
