"""Hand derivation of the 3-species / 2-reaction worked example (toy_3sp_2rx.json).

The paper prints no numeric example, so this toy is worked out by hand here, in
40-digit decimal arithmetic, from the paper's definitions specialised to the toy:

  species X, X2, X3 (W = 10, 20, 30 g/mol), one element; NASA-7 with constant
  cp (a2..a5 = 0), so h/R = a1 T + a6 and s/R = a1 ln T + a7 in closed form
  R1: 2 X + M <=> X2 + M   A = 1e15, b = -1,  E/R = 0,    efficiencies (1, 2, 1)
  R2: X + X2 <=> X3        A = 1e12, b = 0.5, E/R = 5000
  T = 1500 K, P = 1 atm, mole fractions (0.2, 0.5, 0.3), p_ref = 1 bar

  C_k = x_k P / (R T)                                (ideal gas)
  k_f = A T^b exp(-E/(R T))                          (Eq. 5)
  K_c = (p_ref/(R T))^dnu exp(dS/R - dH/(R T))       (Eq. 8, dH and dS taken separately)
  k_r = k_f / K_c                                    (Eq. 7)
  M = sum_k eff_k C_k, multiplying k_f and k_r of R1 (Sec. 2.4)
  q_f = k_f prod C^nu', q_r = k_r prod C^nu''        (Eq. 3)
  omega = nu q_net                                   (Eq. 2)

It imports nothing from the repository.  Run it to rewrite the fixture.
"""
import json
import os
from decimal import Decimal as D, getcontext

getcontext().prec = 40

R = D("8.31446261815324e7")
T = D(1500)
P = D("1.01325e6")
PREF = D("1e6")
x = [D("0.2"), D("0.5"), D("0.3")]
W = [D(10), D(20), D(30)]
a1 = [D("2.5"), D("3.5"), D("4.5")]
a6 = [D(30000), D(0), D(10000)]
a7 = [D(5), D(4), D(3)]


def toy():
    ctot = P / (R * T)
    C = [xi * ctot for xi in x]
    lnT = T.ln()
    h_RT = [a1[k] + a6[k] / T for k in range(3)]
    s_R = [a1[k] * lnT + a7[k] for k in range(3)]
    g_RT = [h_RT[k] - s_R[k] for k in range(3)]
    nu = [[-2, 1, 0], [-1, -1, 1]]
    dH = [sum(n * h for n, h in zip(nu[j], h_RT)) for j in range(2)]
    dS = [sum(n * s for n, s in zip(nu[j], s_R)) for j in range(2)]
    dnu = [sum(nu[j]) for j in range(2)]
    lnKc = [dnu[j] * (PREF / (R * T)).ln() + dS[j] - dH[j] for j in range(2)]
    M = C[0] * 1 + C[1] * 2 + C[2] * 1
    lnkf = [D(10 ** 15).ln() - lnT, D(10 ** 12).ln() + D("0.5") * lnT - D(5000) / T]
    kf = [lnkf[0].exp() * M, lnkf[1].exp()]
    kr = [kf[j] / lnKc[j].exp() for j in range(2)]
    qf = [kf[0] * C[0] * C[0], kf[1] * C[0] * C[1]]
    qr = [kr[0] * C[1], kr[1] * C[2]]
    qn = [qf[j] - qr[j] for j in range(2)]
    omega = [-2 * qn[0] - qn[1], qn[0] - qn[1], qn[1]]
    ymass = [x[k] * W[k] for k in range(3)]
    s = sum(ymass)
    Y = [y / s for y in ymass]
    return dict(c_tot=ctot, C=C, g_RT=g_RT, M=M, lnkf=lnkf, lnKc=lnKc, qf=qf, qr=qr,
                omega=omega, Y=Y, mass_balance=sum(W[k] * omega[k] for k in range(3)))


def main():
    v = toy()
    fmt = (lambda z: [format(e, ".25e") for e in z] if isinstance(z, list) else format(z, ".25e"))
    out = {
        "citation": "hand-worked example of Eqs. 2, 3, 5, 7, 8 and the third-body rule of "
                    "Sec. 2.4; derived by tests/golden/derive_toy.py in 40-digit decimal",
        "mechanism": {
            "species": ["X", "X2", "X3"], "mol_weight": [10.0, 20.0, 30.0],
            "nasa_a1_a6_a7": [[2.5, 30000.0, 5.0], [3.5, 0.0, 4.0], [4.5, 10000.0, 3.0]],
            "reactions": ["2 X + M <=> X2 + M (A=1e15, b=-1, E/R=0, eff=(1,2,1))",
                          "X + X2 <=> X3 (A=1e12, b=0.5, E/R=5000)"],
            "p_ref": 1.0e6, "t_mid": 1000.0,
        },
        "state": {"T": 1500.0, "P": 101325.0e1, "mole_fractions": [0.2, 0.5, 0.3]},
        "expected": {k: fmt(val) for k, val in v.items()},
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "toy_3sp_2rx.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps(out["expected"], indent=1))


if __name__ == "__main__":
    main()
