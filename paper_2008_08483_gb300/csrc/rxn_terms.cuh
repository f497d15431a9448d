// rxn_terms.cuh -- per-reaction rate terms and their temperature derivatives for one
// cell, shared by the derivative kernels (kern_tangent.cu) and the reactor integrator
// (kern_integrate.cu), in double or float arithmetic on the FP64 tables.
//
// For reaction j at temperature T and third-body concentration M:
//   ln k_inf = ln A + b ln T - (E/R) / T,  d ln k_inf / dT = b / T + (E/R) / T^2     (Eq. 5)
//   modifier (Sec. 2.4): third body          ln mod = ln M
//                        Lindemann / Troe    ln mod = ln(Pr / (1 + Pr)) + ln F,
//                                            Pr = k0 M / k_inf
//   k_f = k_inf mod,  k_r = k_f / K_c for reversible reactions                         (Eq. 7)
//   ln K_c and d ln K_c / dT from the folded Gibbs polynomial on
//   [1, ln T, tau, tau^2, tau^3, tau^4, 1/T], tau = T / 1000                          (Eqs. 9-11)
// The Troe factor is the Gilbert-Luther-Troe form (F_cent from three exponentials,
// c = -0.4 - 0.67 log10 F_cent, n = 0.75 - 1.27 log10 F_cent, d = 0.14); its derivatives
// follow by the chain rule.
#pragma once

#include <math.h>

#include "chem_internal.h"

namespace chem {

__device__ __forceinline__ double rt_exp(double x) { return exp(x); }
__device__ __forceinline__ float rt_exp(float x) { return expf(x); }
__device__ __forceinline__ double rt_log(double x) { return log(x); }
__device__ __forceinline__ float rt_log(float x) { return logf(x); }
__device__ __forceinline__ double rt_log10(double x) { return log10(x); }
__device__ __forceinline__ float rt_log10(float x) { return log10f(x); }

template <typename R>
struct RxnTerms {
    R lkinf;      // ln k_inf
    R dlkinf;     // d ln k_inf / dT
    R lmod;       // ln(modifier); 0 for elementary reactions
    R dmod_dlM;   // d ln(modifier) / d ln M at fixed T
    R dmod_dT;    // d ln(modifier) / dT at fixed M
    R lKc;        // ln K_c
    R dlKc;       // d ln K_c / dT
    bool dead;    // k_f = 0: M <= 0 or Pr <= 0
};

// Per-cell temperature features of the rate terms.
template <typename R>
struct TFeat {
    R T, lnT, invT, tau;
    int rg;       // NASA-7 range: 1 when T >= T_mid
};

template <typename R>
__device__ __forceinline__ TFeat<R> t_features(R T, double t_mid)
{
    TFeat<R> f;
    f.T = T;
    f.lnT = rt_log(T);
    f.invT = R(1) / T;
    f.tau = T * R(1e-3);
    f.rg = (double)T >= t_mid ? 1 : 0;
    return f;
}

// M is sum_m eff_m C_m of the reaction (ignored for elementary reactions).
template <typename R>
__device__ __forceinline__ RxnTerms<R> rxn_terms(const RxnF64 *X, const TFeat<R> &tf, R M)
{
    RxnTerms<R> o;
    const R Ti = tf.T, lnT = tf.lnT, invT = tf.invT, tau = tf.tau;
    o.lkinf = R(X->lnA) + R(X->b) * lnT - R(X->EoR) * invT;
    o.dlkinf = R(X->b) * invT + R(X->EoR) * invT * invT;
    o.lmod = 0;
    o.dmod_dlM = 0;
    o.dmod_dT = 0;
    o.dead = false;
    const int kind = X->kind;
    if (kind != 0) {
        if (!(M > R(0))) {
            o.dead = true;
        } else if (kind == 1) {
            o.lmod = rt_log(M);
            o.dmod_dlM = 1;
        } else {
            const R lk0 = R(X->low[0]) + R(X->low[1]) * lnT - R(X->low[2]) * invT;
            const R Pr = rt_exp(lk0 - o.lkinf) * M;
            if (!(Pr > R(0))) {
                o.dead = true;
            } else {
                o.lmod = rt_log(Pr / (R(1) + Pr));
                R dlF_dlPr = 0, dlF_dT = 0;
                if (kind == 3) {
                    const R e3 = rt_exp(-Ti * R(X->troe[2])), e1 = rt_exp(-Ti * R(X->troe[3]));
                    R Fc = R(X->troe[0]) * e3 + R(X->troe[1]) * e1;
                    R dFc = -R(X->troe[0]) * R(X->troe[2]) * e3 - R(X->troe[1]) * R(X->troe[3]) * e1;
                    if (X->troe[4] > 0.0) {
                        const R e2 = rt_exp(-R(X->troe[4]) * invT);
                        Fc += e2;
                        dFc += R(X->troe[4]) * invT * invT * e2;
                    }
                    const R L = rt_log10(Fc);
                    const R dL_dT = dFc / (Fc * R(2.302585092994045684));
                    const R c = R(-0.4) - R(0.67) * L, nn = R(0.75) - R(1.27) * L;
                    const R x = rt_log10(Pr) + c;
                    const R D = nn - R(0.14) * x;
                    const R f1 = x / D, g = R(1) + f1 * f1;
                    o.lmod += L / g * R(2.302585092994045684);
                    dlF_dlPr = -L * R(2) * f1 / (g * g) * (nn / (D * D));
                    const R dD_dL = R(-1.27) + R(0.14) * R(0.67);
                    const R df1_dL = (R(-0.67) * D - x * dD_dL) / (D * D);
                    dlF_dT = (R(1) / g - L * R(2) * f1 / (g * g) * df1_dL) * dL_dT;
                }
                o.dmod_dlM = R(1) / (R(1) + Pr) + dlF_dlPr;
                const R dlPr_dT = (R(X->low[1]) - R(X->b)) * invT +
                                  (R(X->low[2]) - R(X->EoR)) * invT * invT;
                o.dmod_dT = o.dmod_dlM * dlPr_dT + dlF_dT * R(2.302585092994045684);
            }
        }
    }
    const double *kc = X->kc[tf.rg];
    o.lKc = R(kc[0]) + R(kc[1]) * lnT +
            tau * (R(kc[2]) + tau * (R(kc[3]) + tau * (R(kc[4]) + tau * R(kc[5])))) +
            R(kc[6]) * invT;
    o.dlKc = R(kc[1]) * invT +
             (R(kc[2]) + tau * (R(2) * R(kc[3]) + tau * (R(3) * R(kc[4]) + tau * R(4) * R(kc[5])))) *
                 R(1e-3) -
             R(kc[6]) * invT * invT;
    return o;
}

}  // namespace chem
