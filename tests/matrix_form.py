"""The paper's matrix ("exact ANN") form of the source term in dense numpy FP64.

Used by the tests as an independent derivation to pin the loop oracle: the
paper states that its layer form is an exact recasting (Sec. 2.3), so the two
must agree to rounding.  Written from the layer equations:

  ln K_f = X_f W_f + B_f, X_f = [ln T, 1/T], W_f = [beta; -E/R], B_f = ln A   (Eq. 6)
  G = X_G W_G + B_G, X_G = [ln T, T, T^2, T^3, T^4, 1/T]                      (Eq. 10)
  ln K_c = -(X_G W_G' + B_G') nu, with p_ref/(R T) folded into the bias       (Eq. 11)
  M = C E (third-body concentrations, Sec. 2.4)
  Q = exp(ln C nu' + ln K_f) - exp(ln C nu'' + ln K_r), ln K_r = ln K_f - ln K_c  (Eqs. 4, 7)
  Omega = Q_net nu^T                                                           (Eq. 2)

The Gibbs weights follow from g/RT = h/RT - s/R of NASA-7 written on X_G:
W_G rows = [-a1, -a2/2, -a3/6, -a4/12, -a5/20, a6], B_G = a1 - a7.  Folding
ln(p_ref/(R T)) = ln(p_ref/R) - ln T into the layer adds 1 to the ln T row and
-ln(p_ref/R) to the bias.  Falloff reactions are applied elementwise, as the
paper does ("non-matrix", Sec. 2.4).  Requires C > 0.
"""
import numpy as np

R = 8.31446261815324e7


def gibbs_layer(nasa7, p_ref):
    """(W_G' [2, 6, ns], B_G' [2, ns]) per temperature range, p_ref/RT folded in."""
    a = nasa7                                    # [ns, 2, 7]
    W = np.stack([-a[:, :, 0], -a[:, :, 1] / 2, -a[:, :, 2] / 6, -a[:, :, 3] / 12,
                  -a[:, :, 4] / 20, a[:, :, 5]], axis=0)        # [6, ns, 2]
    W = np.transpose(W, (2, 0, 1)).copy()                       # [2, 6, ns]
    B = (a[:, :, 0] - a[:, :, 6]).T.copy()                      # [2, ns]
    W[:, 0, :] += 1.0
    B -= np.log(p_ref / R)
    return W, B


def troe_F(tp, T, Pr):
    alpha, T3, T1, T2 = tp
    Fc = (1 - alpha) * np.exp(-T / T3) + alpha * np.exp(-T / T1)
    if T2 > 0:
        Fc = Fc + np.exp(-T2 / T)
    lFc = np.log10(Fc)
    c = -0.4 - 0.67 * lFc
    n = 0.75 - 1.27 * lFc
    x = np.log10(Pr) + c
    f1 = x / (n - 0.14 * x)
    return 10.0 ** (lFc / (1 + f1 * f1))


def source_term_tc(mech, T, C):
    T = np.asarray(T, float)
    C = np.asarray(C, float)
    nu_f = mech.nu_f.T.astype(float)             # [ns, nr]  (nu')
    nu_r = mech.nu_r.T.astype(float)             # [ns, nr]  (nu'')
    nu = nu_r - nu_f
    Xf = np.stack([np.log(T), 1.0 / T], 1)       # [nc, 2]
    Wf = np.stack([mech.arrh[:, 1], -mech.arrh[:, 2]], 0)
    lnKf = Xf @ Wf + mech.arrh[:, 0][None, :]
    XG = np.stack([np.log(T), T, T**2, T**3, T**4, 1.0 / T], 1)
    WG, BG = gibbs_layer(mech.nasa7, mech.p_ref)
    hi = (T >= mech.t_mid)[:, None]
    G = np.where(hi, XG @ WG[1] + BG[1], XG @ WG[0] + BG[0])   # [nc, ns]
    lnKc = -G @ nu
    kind = mech.kind
    M = C @ mech.eff.T                                         # [nc, nr]
    lnM = np.where((kind == 1)[None, :], np.log(M), 0.0)
    # falloff: ln of k_inf Pr/(1+Pr) F relative to k_inf, elementwise
    lnFall = np.zeros_like(lnKf)
    for j in np.nonzero((kind == 2) | (kind == 3))[0]:
        al = mech.arrh_low[j]
        lnk0 = al[0] + al[1] * np.log(T) - al[2] / T
        Pr = np.exp(lnk0 - lnKf[:, j]) * M[:, j]
        F = troe_F(mech.troe[j], T, Pr) if kind[j] == 3 else 1.0
        lnFall[:, j] = np.log(Pr / (1 + Pr) * F)
    lnKf_eff = lnKf + lnM + lnFall
    lnKr = lnKf_eff - lnKc
    lnC = np.log(C)
    Qf = np.exp(lnC @ nu_f + lnKf_eff)
    Qr = np.exp(lnC @ nu_r + lnKr) * mech.reversible[None, :]
    return (Qf - Qr) @ nu.T
