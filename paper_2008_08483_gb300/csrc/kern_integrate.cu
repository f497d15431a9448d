// kern_integrate.cu -- constant-pressure adiabatic 0-D reactors: right-hand side, analytic
// Jacobian and a batched Rosenbrock integrator, one warp per cell, FP64.
//
// Reactor (state y = (T, Y_1..Y_ns), pressure P fixed per cell):
//   S = sum_k Y_k / W_k,  rho = P / (R T S),  C_k = rho Y_k / W_k
//   dY_k/dt = W_k omega_k / rho,   dT/dt = -Q / (rho c_p),
//   Q = sum_k H_k omega_k, H_k = R T (h/RT)_k, c_p = R sum_k Y_k (cp/R)_k / W_k   (Eq. 10)
// omega (Eqs. 2-8, Sec. 2.4) with q_f = k_f prod_k C_k^nu'_k and q_r = k_r prod_k C_k^nu''_k
// as products (not logarithms), so that d q / dC_m needs no division by C_m and C_m = 0
// is an ordinary point:
//   d q_f / dC_m = k_f nu'_m C_m^(nu'_m - 1) prod_{k != m} C_k^nu'_k + (d k_f / dM) eff_m prod C^nu'
// and d k_f / dM = k_f (d ln mod / d ln M) / M, so the third-body part of d q_net / dC_m is
// eff_m q_net (d ln mod / d ln M) / M.  The rate terms and their temperature derivatives
// are the ones of the derivative kernels (rxn_terms.cuh).  The Jacobian in (T, Y) follows
// from d omega / dC and d omega / dT|_C by the chain rule through C(T, Y):
//   dC_m/dT = -C_m/T,  dC_m/dY_n = rho delta_mn / W_m - C_m / (S W_n),
//   d(1/rho)/dT = 1/(rho T),  d(1/rho)/dY_n = 1/(rho S W_n).
//
// Work split inside a warp.  Per 32 reactions, each lane evaluates one reaction's scalars
// (k_f, k_r, q_net, d q_net/dT, d q_net/dM); the warp then walks those 32 reactions in
// order, broadcasting the scalars with shuffles, and the lanes apply one reaction's
// updates to distinct entries (rows for omega, row x column pairs for d omega / dC).  The
// accumulation order is therefore fixed: results are deterministic and independent of
// which warp or batch a cell is in.
//
// Integrator: Rodas3 (Sandu, Verwer, Blom, Spee, Carmichael, Potra, "Benchmarking stiff
// ODE solvers for atmospheric chemistry problems II: Rosenbrock solvers", Atmos. Environ.
// 31 (1997)), four stages, order 3, embedded order 2, stiffly accurate, L-stable; used in
// the form without Jacobian-vector products (Hairer & Wanner, Solving ODEs II, Sec. IV.7):
//   (I / (h gamma) - J) U_i = f(y + sum_j a_ij U_j) + sum_j (c_ij / h) U_j
//   y_new = y + sum_i m_i U_i,   err = sum_i e_i U_i
// with (a, c, m, e) computed on the host from the classical table (alpha, gamma, b, bhat).
// The right-hand side, the LU (partial pivoting), the solves and the error control are
// FP64; the stage Jacobian J is FP64 too unless the caller asks for it in FP32
// (reactor_jac_f32): J enters only the stage matrix, so an FP32 J changes the step's
// arithmetic but not what the error control checks.  Step size: RMS error norm
// with weights atol + rtol max(|y|, |y_new|), factor 0.9 err^(-1/3) clamped to [0.2, 5],
// no growth right after a rejection; or, on request, a fixed number of equal steps without
// error control (the L-stable step of an operator-split CFD solver).
#include <math.h>
#include <string.h>

#include <mutex>

#include "chem_internal.h"
#include "rxn_terms.cuh"

namespace chem {

// ---------------------------------------------------------------------------------------
// method coefficients
// ---------------------------------------------------------------------------------------

constexpr int kStages = 4;
constexpr int kDStride = kIntMax + 1;

// classical Rodas3 table
static const double kGammaII = 0.5;
static const double kAlpha[4][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}, {1, 0, 0, 0}, {0.75, -0.25, 0.5, 0}};
static const double kGammaIJ[4][4] = {
    {0, 0, 0, 0}, {1, 0, 0, 0}, {-0.25, -0.25, 0, 0}, {1.0 / 12, 1.0 / 12, -2.0 / 3, 0}};
static const double kB[4] = {5.0 / 6, -1.0 / 6, -1.0 / 6, 0.5};
static const double kBhat[4] = {0.75, -0.25, 0.5, 0};

struct RosCoef {
    double gamma;
    double a[4][4], c[4][4];
    double m[4], e[4];
};

// Gamma = (gamma_ij) with gamma_ii on the diagonal; a = alpha Gamma^-1,
// c = diag(1/gamma_ii) - Gamma^-1, m = b Gamma^-1, e = (b - bhat) Gamma^-1.
static RosCoef make_coef()
{
    double G[4][4], Gi[4][4];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) G[i][j] = i == j ? kGammaII : (j < i ? kGammaIJ[i][j] : 0.0);
    // inverse of the lower-triangular Gamma by forward substitution, column by column
    for (int col = 0; col < 4; ++col)
        for (int i = 0; i < 4; ++i) {
            double s = i == col ? 1.0 : 0.0;
            for (int j = 0; j < i; ++j) s -= G[i][j] * Gi[j][col];
            Gi[i][col] = s / G[i][i];
        }
    RosCoef r;
    memset(&r, 0, sizeof r);
    r.gamma = kGammaII;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            double s = 0.0;
            for (int k = 0; k < 4; ++k) s += kAlpha[i][k] * Gi[k][j];
            r.a[i][j] = j < i ? s : 0.0;
            r.c[i][j] = j < i ? -Gi[i][j] : 0.0;
        }
    for (int j = 0; j < 4; ++j) {
        double sm = 0.0, se = 0.0;
        for (int k = 0; k < 4; ++k) {
            sm += kB[k] * Gi[k][j];
            se += (kB[k] - kBhat[k]) * Gi[k][j];
        }
        r.m[j] = sm;
        r.e[j] = se;
    }
    return r;
}

// ---------------------------------------------------------------------------------------
// per-warp workspace layout (offsets in doubles from the warp's base)
// ---------------------------------------------------------------------------------------

struct WarpLayout {
    int n, ldw;          // system size ns + 1; leading dimension of the matrix (odd)
    int nv, nsp;         // padded vector lengths
    int oY, oYs, oR, oU, oYn, oInvd, oPiv;    // vectors; U holds kStages vectors
    int oC, oH, oCp, oDcp, oWo, oJT, oVM, oWC, oAK;   // per-species arrays
    int oD;              // [32][kDStride] per-column derivatives of one group of reactions
    int oQ;              // [3][32] q_net, d q_net/dT, d q_net/dM of one group
    int oMat;            // matrix offset when it lives in shared memory, else -1
    int per_warp;        // doubles of shared memory per warp
};

static WarpLayout make_layout(int ns, bool mat_in_smem)
{
    WarpLayout L;
    L.n = ns + 1;
    L.ldw = L.n | 1;
    L.nv = (L.n + 1) & ~1;
    L.nsp = (ns + 1) & ~1;
    int o = 0;
    L.oY = o; o += L.nv;
    L.oYs = o; o += L.nv;
    L.oR = o; o += L.nv;
    L.oU = o; o += kStages * L.nv;
    L.oYn = o; o += L.nv;
    L.oInvd = o; o += L.nv;
    L.oPiv = o; o += L.nv;            // 2 nv ints: piv, then the combined permutation
    L.oC = o; o += L.nsp;
    L.oH = o; o += L.nsp;
    L.oCp = o; o += L.nsp;
    L.oDcp = o; o += L.nsp;
    L.oWo = o; o += L.nsp;
    L.oJT = o; o += L.nsp;
    L.oVM = o; o += L.nsp;
    L.oWC = o; o += L.nsp;
    L.oAK = o; o += L.nsp;
    L.oD = o; o += 32 * kDStride;
    L.oQ = o; o += 96;
    if (mat_in_smem) {
        L.oMat = o;
        o += L.n * L.ldw;
        o = (o + 1) & ~1;
    } else {
        L.oMat = -1;
    }
    L.per_warp = o;
    return L;
}

struct IntegParams {
    int64_t n;
    const double *T, *P, *Y;  // inputs (ode_rhs / jacobian) or in/out state (integrate)
    double *Tout, *Yout;
    int64_t ldY;
    double *f;                // ode_rhs output
    int64_t ldF;
    double *J;                // ode_jacobian output
    double t_end, rtol, atol, h0, hmin, hmax, ign_dT;
    int64_t max_steps;
    int fixed_steps;          // > 0: this many equal steps, no error control
    int jac32;                // integrate: stage Jacobian in FP32 (else FP64)
    int32_t *status, *nacc, *nrej;
    double *t_ign;
    const int64_t *n_dev;     // integrate: cell count read on the device (NULL: use n)
    unsigned int *queue;      // [0] next cell, [1] failed cells
    double *gmat;             // per-warp matrices when they do not fit in shared memory
    WarpLayout L;
    RosCoef rc;
};

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double ipow(double c, int e)
{
    double p = 1.0;
    for (int t = 0; t < e; ++t) p *= c;
    return p;
}

struct Ctx {
    double *y, *ys, *r, *U, *yn, *invd;
    int *piv, *pv;
    double *C, *H, *Cp, *Dcp, *Wo, *JT, *VM, *WC, *AK, *D, *Q;
    double *A;                // matrix, row-major with leading dimension ldw
};

__device__ __forceinline__ Ctx make_ctx(double *base, double *mat, const WarpLayout &L)
{
    Ctx c;
    c.y = base + L.oY;
    c.ys = base + L.oYs;
    c.r = base + L.oR;
    c.U = base + L.oU;
    c.yn = base + L.oYn;
    c.invd = base + L.oInvd;
    c.piv = (int *)(base + L.oPiv);
    c.pv = c.piv + L.nv;
    c.C = base + L.oC;
    c.H = base + L.oH;
    c.Cp = base + L.oCp;
    c.Dcp = base + L.oDcp;
    c.Wo = base + L.oWo;
    c.JT = base + L.oJT;
    c.VM = base + L.oVM;
    c.WC = base + L.oWC;
    c.AK = base + L.oAK;
    c.D = base + L.oD;
    c.Q = base + L.oQ;
    c.A = mat;
    return c;
}

__device__ void jac_finish(const MechViewF64 &mv, const IntView &iv, const WarpLayout &L,
                           const Ctx &c, const double *ys, double T, double S, double rho,
                           double rc, double Q, int lane);

// f(ys) into fo; with JAC also the Jacobian into c.A (row-major, ldw).
template <bool JAC>
__device__ void reactor_eval(const MechViewF64 &mv, const IntView &iv, const WarpLayout &L,
                             const Ctx &c, double P, const double *ys, double *fo, int lane)
{
    const int ns = mv.ns, ldw = L.ldw;
    const double T = ys[0];
    double s = 0.0;
    for (int k = lane; k < ns; k += 32) s += ys[1 + k] * mv.invW[k];
    const double S = warp_sum(s);
    const double rho = P / (kR * T * S);
    const TFeat<double> tf = t_features<double>(T, mv.t_mid);
    for (int k = lane; k < ns; k += 32) {
        c.C[k] = rho * ys[1 + k] * mv.invW[k];
        const double *a = iv.nasa + (size_t)k * 14 + tf.rg * 7;
        c.Cp[k] = a[0] + T * (a[1] + T * (a[2] + T * (a[3] + T * a[4])));
        c.H[k] = a[0] + T * (a[1] * 0.5 + T * (a[2] * (1.0 / 3) + T * (a[3] * 0.25 + T * a[4] * 0.2))) +
                 a[5] / T;
        c.Wo[k] = 0.0;
        if (JAC) {
            c.Dcp[k] = kR * (a[1] + T * (2.0 * a[2] + T * (3.0 * a[3] + T * 4.0 * a[4])));
            c.JT[k] = 0.0;
            c.VM[k] = 0.0;
        }
    }
    if (JAC) {
        for (int k = 0; k < ns; ++k)
            for (int m = lane; m < ns; m += 32) c.A[(1 + k) * ldw + 1 + m] = 0.0;
    }
    __syncwarp();
    const double ctot = P / (kR * T);     // sum_k C_k
    for (int g = 0; g < iv.n_slots; g += 32) {
        // phase A: one reaction per lane (all lanes of a group share the reaction kind)
        const int j = iv.order[g + lane];
        double qn = 0.0, dqT = 0.0, dqM = 0.0;
        if (j >= 0) {
            const RxnF64 *X = mv.rxn + j;
            double M = 1.0;
            if (X->kind != 0) {
                M = ctot;
                for (int t = X->tb_begin; t < X->tb_end; ++t) M += mv.tb_e[t] * c.C[mv.tb_sp[t]];
            }
            const RxnTerms<double> rt = rxn_terms<double>(X, tf, M);
            double kf = 0.0, kr = 0.0;
            if (!rt.dead) {
                kf = exp(rt.lkinf + rt.lmod);
                kr = X->rev ? exp(rt.lkinf + rt.lmod - rt.lKc) : 0.0;
                double pf = kf, pr = kr;
                for (int t = 0; t < X->nf; ++t) pf *= ipow(c.C[X->spf[t]], X->nuf[t]);
                if (X->rev)
                    for (int t = 0; t < X->nr; ++t) pr *= ipow(c.C[X->spr[t]], X->nur[t]);
                qn = pf - pr;
                if (JAC) {
                    const double dlkf = rt.dlkinf + rt.dmod_dT;
                    dqT = pf * dlkf - pr * (dlkf - rt.dlKc);
                    if (X->kind != 0) dqM = qn * rt.dmod_dlM / M;
                }
            }
            if (JAC) {
                // mass-action part of d q_net / dC_m for each column m of the reaction:
                // k_f nu'_m C_m^(nu'_m - 1) prod_{u != m} C_u^nu'_u - (same for the reverse)
                const RxnInt *I = iv.rxn + j;
                const int ncol = I->ncol;
                for (int cc = 0; cc < ncol; ++cc) {
                    const int ef = I->col_nuf[cc], er = I->col_nur[cc];
                    const double cm = c.C[I->col_sp[cc]];
                    double df = 0.0, dr = 0.0;
                    if (ef) df = kf * (double)ef * ipow(cm, ef - 1);
                    if (er && kr != 0.0) dr = kr * (double)er * ipow(cm, er - 1);
                    for (int u = 0; u < ncol; ++u) {
                        if (u == cc) continue;
                        const double cu = c.C[I->col_sp[u]];
                        if (I->col_nuf[u]) df *= ipow(cu, I->col_nuf[u]);
                        if (I->col_nur[u]) dr *= ipow(cu, I->col_nur[u]);
                    }
                    c.D[lane * kDStride + cc] = df - dr;
                }
            }
        }
        c.Q[lane] = qn;
        if (JAC) {
            c.Q[32 + lane] = dqT;
            c.Q[64 + lane] = dqM;
        }
        __syncwarp();
        // phase B: each lane gathers the group's contributions to its own species rows
        // (fixed order: slot order within the group), so no two lanes touch one entry
        const int *gp = iv.gptr + (g >> 5) * (ns + 1);
        for (int k = lane; k < ns; k += 32) {
            const int e0 = gp[k], e1 = gp[k + 1];
            double w = 0.0, jt = 0.0, vm = 0.0;
            for (int e = e0; e < e1; ++e) {
                const int r = iv.gent_slot[e];
                const double nu = iv.gent_nu[e];
                w += nu * c.Q[r];
                if (JAC) {
                    jt += nu * c.Q[32 + r];
                    vm += nu * c.Q[64 + r];
                }
            }
            c.Wo[k] += w;
            if (JAC) {
                c.JT[k] += jt;
                c.VM[k] += vm;
                double *Ak = c.A + (1 + k) * ldw + 1;
                for (int e = e0; e < e1; ++e) {
                    const int r = iv.gent_slot[e];
                    const double nu = iv.gent_nu[e];
                    const int jr = iv.order[g + r];
                    const RxnInt *I = iv.rxn + jr;
                    const int ncol = I->ncol;
                    for (int cc = 0; cc < ncol; ++cc) Ak[I->col_sp[cc]] += nu * c.D[r * kDStride + cc];
                    // listed third-body efficiencies: (eff_m - 1) part of d q_net / dC_m
                    const double dm = c.Q[64 + r];
                    if (dm != 0.0) {
                        const RxnF64 *X = mv.rxn + jr;
                        const double s = nu * dm;
                        for (int t = X->tb_begin; t < X->tb_end; ++t) Ak[mv.tb_sp[t]] += s * mv.tb_e[t];
                    }
                }
            }
        }
        __syncwarp();
    }
    __syncwarp();
    // right-hand side
    double cp = 0.0, q = 0.0;
    for (int k = lane; k < ns; k += 32) {
        cp += ys[1 + k] * c.Cp[k] * mv.invW[k];
        q += c.H[k] * c.Wo[k];
    }
    cp = warp_sum(cp) * kR;               // erg / (g K)
    const double Q = warp_sum(q) * kR * T;
    const double rc = rho * cp;
    if (lane == 0) fo[0] = -Q / rc;
    for (int k = lane; k < ns; k += 32) fo[1 + k] = iv.W[k] * c.Wo[k] / rho;
    if constexpr (JAC) jac_finish(mv, iv, L, c, ys, T, S, rho, rc, Q, lane);
    __syncwarp();
}

// The (T, Y) Jacobian of the reactor from the accumulated d omega / dC (in c.A), d omega / dT
// at fixed C (c.JT) and the column-constant third-body part (c.VM); see the file comment.
__device__ void jac_finish(const MechViewF64 &mv, const IntView &iv, const WarpLayout &L,
                           const Ctx &c, const double *ys, double T, double S, double rho,
                           double rc, double Q, int lane)
{
    const int ns = mv.ns, ldw = L.ldw;
    // d omega / dC: add the column-constant part (efficiency 1 of every species in M)
    for (int k = 0; k < ns; ++k) {
        const double v = c.VM[k];
        for (int m = lane; m < ns; m += 32) c.A[(1 + k) * ldw + 1 + m] += v;
    }
    __syncwarp();
    const double invS = 1.0 / S;
    double hw = 0.0, dqt = 0.0, dcpt = 0.0;
    for (int k = lane; k < ns; k += 32) {
        double w = 0.0;
        for (int m = 0; m < ns; ++m) w += c.A[(1 + k) * ldw + 1 + m] * c.C[m];
        c.WC[k] = w;                                       // sum_m d omega_k/dC_m C_m
        const double dwT = c.JT[k] - w / T;                // d omega_k / dT along C(T, Y)
        c.JT[k] = dwT;
        c.AK[k] = iv.W[k] * (c.Wo[k] - w) * invS / rho;
        hw += c.H[k] * w;
        dqt += c.Cp[k] * c.Wo[k] + T * c.H[k] * dwT;
        dcpt += ys[1 + k] * c.Dcp[k] * mv.invW[k];
    }
    hw = warp_sum(hw);
    dqt = warp_sum(dqt) * kR;
    dcpt = warp_sum(dcpt);
    __syncwarp();
    // Y columns: in-place transform of d omega / dC, and the T row entry of each column
    for (int m = lane; m < ns; m += 32) {
        const double iWm = mv.invW[m];
        double hs = 0.0;
        for (int k = 0; k < ns; ++k) {
            double *e = c.A + (1 + k) * ldw + 1 + m;
            const double jc = *e;
            hs += c.H[k] * jc;
            *e = iv.W[k] * iWm * jc + c.AK[k] * iWm;
        }
        const double dQ = kR * T * (rho * iWm * hs - invS * iWm * hw);
        const double drc = -rc * invS * iWm + rho * kR * c.Cp[m] * iWm;
        c.A[1 + m] = -dQ / rc + Q * drc / (rc * rc);
    }
    // T column
    for (int k = lane; k < ns; k += 32)
        c.A[(1 + k) * ldw] = iv.W[k] * c.JT[k] / rho + iv.W[k] * c.Wo[k] / (rho * T);
    if (lane == 0) {
        const double drcT = -rc / T + rho * dcpt;
        c.A[0] = -dqt / rc + Q * drcT / (rc * rc);
    }
    __syncwarp();
}

// ---------------------------------------------------------------------------------------
// The stage Jacobian in FP32 (on request).  The integrator's right-hand side, LU, solves and
// error control stay FP64; the Jacobian only enters the stage matrix (I / (h gamma) - J), and
// here it is evaluated in FP32 with the structure of reactor_eval<true> and jac_finish: float scratch
// laid over the warp's double scratch arrays, and a float matrix over the first half of the
// matrix storage, widened to double in place at the end.  The mass-action products and their
// column derivatives are formed from ln C (once per species): d q_f / dC_m = nu'_m q_f / C_m
// for C_m > 0, and for C_m <= 0 (only nu'_m = 1 contributes) k_f prod_{u != m} C_u^nu'_u; the
// exponentials are clamped below the float overflow, so k_r, which can exceed the float
// range where the reverse products are tiny, is never formed on its own.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ float warp_sumf(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float exp_clamped(float x) { return expf(fminf(x, 88.0f)); }

// float views of the warp's double scratch (each double array holds twice as many floats)
struct CtxF {
    float *C, *lnC, *H, *Cp, *Dcp, *Wo, *JT, *VM, *WC, *AK, *D, *Q, *A;
};

__device__ __forceinline__ CtxF ctx_f32(const Ctx &c, const WarpLayout &L)
{
    CtxF f;
    f.C = (float *)c.C;
    f.lnC = f.C + L.nsp;
    f.H = (float *)c.H;
    f.Cp = (float *)c.Cp;
    f.Dcp = (float *)c.Dcp;
    f.Wo = (float *)c.Wo;
    f.JT = (float *)c.JT;
    f.VM = (float *)c.VM;
    f.WC = (float *)c.WC;
    f.AK = (float *)c.AK;
    f.D = (float *)c.D;
    f.Q = (float *)c.Q;
    f.A = (float *)c.A;
    return f;
}

// d q / dC_m of one side of reaction I at column cc: nu_m prod C^nu / C_m from the side's
// log-product Ls (which includes nu_m ln C_m), or, when C_m <= 0 and nu_m = 1, the product
// of the side's other factors
__device__ __forceinline__ float side_deriv(const RxnInt *I, const float *lnC, int cc, bool fwd,
                                            float lk, float Ls, bool zero_other)
{
    const int nu = fwd ? I->col_nuf[cc] : I->col_nur[cc];
    if (!nu) return 0.0f;
    const float l = lnC[I->col_sp[cc]];
    if (l > -INFINITY) return zero_other ? 0.0f : (float)nu * exp_clamped(Ls - l);
    if (nu != 1) return 0.0f;
    float Lo = lk;
    for (int u = 0; u < I->ncol; ++u) {
        const int nuu = fwd ? I->col_nuf[u] : I->col_nur[u];
        if (u == cc || !nuu) continue;
        const float lu = lnC[I->col_sp[u]];
        if (!(lu > -INFINITY)) return 0.0f;
        Lo += (float)nuu * lu;
    }
    return exp_clamped(Lo);
}

// The (T, Y) Jacobian of the reactor at ys in FP32, into c.A (double, row-major, ldw).
__device__ void reactor_jac_f32(const MechViewF64 &mv, const IntView &iv, const WarpLayout &L,
                                const Ctx &c, double Pd, const double *ys, int lane)
{
    const int ns = mv.ns, ldw = L.ldw;
    const CtxF f = ctx_f32(c, L);
    const float kRf = (float)kR;
    const float T = (float)ys[0], P = (float)Pd;
    float s = 0.0f;
    for (int k = lane; k < ns; k += 32) s += (float)ys[1 + k] * (float)mv.invW[k];
    const float S = warp_sumf(s);
    const float rho = P / (kRf * T * S);
    const TFeat<float> tf = t_features<float>(T, mv.t_mid);
    for (int k = lane; k < ns; k += 32) {
        const float Ck = rho * (float)ys[1 + k] * (float)mv.invW[k];
        f.C[k] = Ck;
        f.lnC[k] = Ck > 0.0f ? logf(Ck) : -INFINITY;
        const double *a = iv.nasa + (size_t)k * 14 + tf.rg * 7;
        const float a0 = (float)a[0], a1 = (float)a[1], a2 = (float)a[2], a3 = (float)a[3],
                    a4 = (float)a[4], a5 = (float)a[5];
        f.Cp[k] = a0 + T * (a1 + T * (a2 + T * (a3 + T * a4)));
        f.H[k] = a0 + T * (a1 * 0.5f + T * (a2 * (1.0f / 3) + T * (a3 * 0.25f + T * a4 * 0.2f))) + a5 / T;
        f.Dcp[k] = kRf * (a1 + T * (2.0f * a2 + T * (3.0f * a3 + T * 4.0f * a4)));
        f.Wo[k] = 0.0f;
        f.JT[k] = 0.0f;
        f.VM[k] = 0.0f;
    }
    for (int k = 0; k < ns; ++k)
        for (int m = lane; m < ns; m += 32) f.A[(1 + k) * ldw + 1 + m] = 0.0f;
    __syncwarp();
    const float ctot = P / (kRf * T);
    for (int g = 0; g < iv.n_slots; g += 32) {
        // phase A: one reaction per lane
        const int j = iv.order[g + lane];
        float qn = 0.0f, dqT = 0.0f, dqM = 0.0f;
        if (j >= 0) {
            const RxnF64 *X = mv.rxn + j;
            const RxnInt *I = iv.rxn + j;
            const int ncol = I->ncol;
            float M = 1.0f;
            if (X->kind != 0) {
                M = ctot;
                for (int t = X->tb_begin; t < X->tb_end; ++t) M += (float)mv.tb_e[t] * f.C[mv.tb_sp[t]];
            }
            const RxnTerms<float> rt = rxn_terms<float>(X, tf, M);
            float *Dl = f.D + lane * kDStride;
            if (!rt.dead) {
                const float lkf = rt.lkinf + rt.lmod, lkr = lkf - rt.lKc;
                float Lf = lkf, Lr = lkr;
                bool zf = false, zr = false;
                for (int cc = 0; cc < ncol; ++cc) {
                    const float l = f.lnC[I->col_sp[cc]];
                    const int ef = I->col_nuf[cc], er = I->col_nur[cc];
                    if (ef) {
                        if (l > -INFINITY) Lf += (float)ef * l;
                        else zf = true;
                    }
                    if (er) {
                        if (l > -INFINITY) Lr += (float)er * l;
                        else zr = true;
                    }
                }
                const bool rev = X->rev != 0;
                const float pf = zf ? 0.0f : exp_clamped(Lf);
                const float pr = (!rev || zr) ? 0.0f : exp_clamped(Lr);
                qn = pf - pr;
                const float dlkf = rt.dlkinf + rt.dmod_dT;
                dqT = pf * dlkf - pr * (dlkf - rt.dlKc);
                if (X->kind != 0) dqM = qn * rt.dmod_dlM / M;
                for (int cc = 0; cc < ncol; ++cc) {
                    const float df = side_deriv(I, f.lnC, cc, true, lkf, Lf, zf);
                    const float dr = rev ? side_deriv(I, f.lnC, cc, false, lkr, Lr, zr) : 0.0f;
                    Dl[cc] = df - dr;
                }
            } else {
                for (int cc = 0; cc < ncol; ++cc) Dl[cc] = 0.0f;
            }
        }
        f.Q[lane] = qn;
        f.Q[32 + lane] = dqT;
        f.Q[64 + lane] = dqM;
        __syncwarp();
        // phase B: each lane gathers the group's contributions to its own species rows
        const int *gp = iv.gptr + (g >> 5) * (ns + 1);
        for (int k = lane; k < ns; k += 32) {
            const int e0 = gp[k], e1 = gp[k + 1];
            float w = 0.0f, jt = 0.0f, vm = 0.0f;
            float *Ak = f.A + (1 + k) * ldw + 1;
            for (int e = e0; e < e1; ++e) {
                const int r = iv.gent_slot[e];
                const float nu = (float)iv.gent_nu[e];
                w += nu * f.Q[r];
                jt += nu * f.Q[32 + r];
                vm += nu * f.Q[64 + r];
                const int jr = iv.order[g + r];
                const RxnInt *I = iv.rxn + jr;
                const int ncol = I->ncol;
                for (int cc = 0; cc < ncol; ++cc) Ak[I->col_sp[cc]] += nu * f.D[r * kDStride + cc];
                const float dm = f.Q[64 + r];
                if (dm != 0.0f) {
                    const RxnF64 *X = mv.rxn + jr;
                    const float sm = nu * dm;
                    for (int t = X->tb_begin; t < X->tb_end; ++t) Ak[mv.tb_sp[t]] += sm * (float)mv.tb_e[t];
                }
            }
            f.Wo[k] += w;
            f.JT[k] += jt;
            f.VM[k] += vm;
        }
        __syncwarp();
    }
    __syncwarp();
    // heat release and heat capacity (as the right-hand side), then jac_finish's chain rule
    float cp = 0.0f, q = 0.0f;
    for (int k = lane; k < ns; k += 32) {
        cp += (float)ys[1 + k] * f.Cp[k] * (float)mv.invW[k];
        q += f.H[k] * f.Wo[k];
    }
    cp = warp_sumf(cp) * kRf;
    const float Qh = warp_sumf(q) * kRf * T;
    const float rc = rho * cp;
    for (int k = 0; k < ns; ++k) {
        const float v = f.VM[k];
        for (int m = lane; m < ns; m += 32) f.A[(1 + k) * ldw + 1 + m] += v;
    }
    __syncwarp();
    const float invS = 1.0f / S;
    float hw = 0.0f, dqt = 0.0f, dcpt = 0.0f;
    for (int k = lane; k < ns; k += 32) {
        float w = 0.0f;
        for (int m = 0; m < ns; ++m) w += f.A[(1 + k) * ldw + 1 + m] * f.C[m];
        f.WC[k] = w;
        const float dwT = f.JT[k] - w / T;
        f.JT[k] = dwT;
        f.AK[k] = (float)iv.W[k] * (f.Wo[k] - w) * invS / rho;
        hw += f.H[k] * w;
        dqt += f.Cp[k] * f.Wo[k] + T * f.H[k] * dwT;
        dcpt += (float)ys[1 + k] * f.Dcp[k] * (float)mv.invW[k];
    }
    hw = warp_sumf(hw);
    dqt = warp_sumf(dqt) * kRf;
    dcpt = warp_sumf(dcpt);
    __syncwarp();
    for (int m = lane; m < ns; m += 32) {
        const float iWm = (float)mv.invW[m];
        float hs = 0.0f;
        for (int k = 0; k < ns; ++k) {
            float *e = f.A + (1 + k) * ldw + 1 + m;
            const float jc = *e;
            hs += f.H[k] * jc;
            *e = (float)iv.W[k] * iWm * jc + f.AK[k] * iWm;
        }
        const float dQ = kRf * T * (rho * iWm * hs - invS * iWm * hw);
        const float drc = -rc * invS * iWm + rho * kRf * f.Cp[m] * iWm;
        f.A[1 + m] = -dQ / rc + Qh * drc / (rc * rc);
    }
    for (int k = lane; k < ns; k += 32)
        f.A[(1 + k) * ldw] = (float)iv.W[k] * f.JT[k] / rho + (float)iv.W[k] * f.Wo[k] / (rho * T);
    if (lane == 0) {
        const float drcT = -rc / T + rho * dcpt;
        f.A[0] = -dqt / rc + Qh * drcT / (rc * rc);
    }
    __syncwarp();
    // widen in place, from the end: double i covers floats 2i and 2i + 1, which (for i >= 1)
    // lie above float i, so every float is read (by the whole warp, before a write) ahead of
    // the write that covers it
    const int tot = L.n * ldw;
    for (int base = tot - 1; base >= 0; base -= 32) {
        const int i = base - lane;
        const float v = i >= 0 ? f.A[i] : 0.0f;
        __syncwarp();
        if (i >= 0) c.A[i] = (double)v;
        __syncwarp();
    }
}

// In-place LU with partial pivoting of the n x n matrix A (leading dimension ldw); unit
// lower L below the diagonal, U on and above it, 1/U_kk in invd, row interchanges in piv
// and their combined permutation in pv ((P b)_i = b_{pv_i}).  False if a pivot is zero or
// not finite.
__device__ bool lu_factor(const Ctx &c, int n, int ldw, int lane)
{
    double *A = c.A;
    for (int k = 0; k < n; ++k) {
        double best = -1.0;
        int bi = k;
        for (int i = k + lane; i < n; i += 32) {
            const double v = fabs(A[i * ldw + k]);
            if (v > best) {
                best = v;
                bi = i;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) {
                best = ob;
                bi = oi;
            }
        }
        if (!(best > 0.0) || !isfinite(best)) return false;
        if (bi != k)
            for (int col = lane; col < n; col += 32) {
                const double t = A[k * ldw + col];
                A[k * ldw + col] = A[bi * ldw + col];
                A[bi * ldw + col] = t;
            }
        if (lane == 0) c.piv[k] = bi;
        __syncwarp();
        const double inv = 1.0 / A[k * ldw + k];
        if (lane == 0) c.invd[k] = inv;
        for (int i = k + 1 + lane; i < n; i += 32) A[i * ldw + k] *= inv;
        __syncwarp();
        for (int jc = k + 1 + lane; jc < n; jc += 32) {
            const double u = A[k * ldw + jc];
            int i = k + 1;
            for (; i + 7 < n; i += 8) {            // 8 rows per batch: loads issue together
                double a[8], b[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    a[q] = A[(i + q) * ldw + k];
                    b[q] = A[(i + q) * ldw + jc];
                }
#pragma unroll
                for (int q = 0; q < 8; ++q) A[(i + q) * ldw + jc] = b[q] - a[q] * u;
            }
            for (; i < n; ++i) A[i * ldw + jc] -= A[i * ldw + k] * u;
        }
        __syncwarp();
    }
    if (lane == 0) {
        for (int i = 0; i < n; ++i) c.pv[i] = i;
        for (int k = 0; k < n; ++k) {
            const int p = c.piv[k];
            const int t = c.pv[k];
            c.pv[k] = c.pv[p];
            c.pv[p] = t;
        }
    }
    __syncwarp();
    return true;
}

// x = A^-1 b for the factors of lu_factor; b is read from rhs, x written to x (distinct).
// Systems of up to 64 unknowns keep x in registers (two per lane) and broadcast each solved
// component with a shuffle; larger ones work in shared memory.
__device__ void lu_solve(const Ctx &c, int n, int ldw, const double *rhs, double *x, int lane)
{
    const double *A = c.A;
    if (n <= 64) {
        const int i0 = lane, i1 = lane + 32;
        double x0 = i0 < n ? rhs[c.pv[i0]] : 0.0;
        double x1 = i1 < n ? rhs[c.pv[i1]] : 0.0;
        for (int j = 0; j < n - 1; ++j) {
            const double xj = __shfl_sync(0xffffffffu, j < 32 ? x0 : x1, j & 31);
            if (i0 > j && i0 < n) x0 -= A[i0 * ldw + j] * xj;
            if (i1 > j && i1 < n) x1 -= A[i1 * ldw + j] * xj;
        }
        for (int j = n - 1; j >= 0; --j) {
            const double xj = __shfl_sync(0xffffffffu, j < 32 ? x0 : x1, j & 31) * c.invd[j];
            if (i0 < j) x0 -= A[i0 * ldw + j] * xj;
            else if (i0 == j) x0 = xj;
            if (i1 < j) x1 -= A[i1 * ldw + j] * xj;
            else if (i1 == j) x1 = xj;
        }
        if (i0 < n) x[i0] = x0;
        if (i1 < n) x[i1] = x1;
        __syncwarp();
        return;
    }
    for (int i = lane; i < n; i += 32) x[i] = rhs[c.pv[i]];
    __syncwarp();
    for (int j = 0; j < n - 1; ++j) {
        const double xj = x[j];
        for (int i = j + 1 + lane; i < n; i += 32) x[i] -= A[i * ldw + j] * xj;
        __syncwarp();
    }
    for (int j = n - 1; j >= 0; --j) {
        const double xj = x[j] * c.invd[j];
        for (int i = lane; i < j; i += 32) x[i] -= A[i * ldw + j] * xj;
        __syncwarp();
        if (lane == 0) x[j] = xj;
        __syncwarp();
    }
}

enum IntegMode { kModeRhs = 0, kModeJac = 1, kModeIntegrate = 2 };

template <int MODE>
__global__ void __launch_bounds__(256) k_reactor(MechViewF64 mv, IntView iv, IntegParams p)
{
    extern __shared__ double smem_int[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    const WarpLayout &L = p.L;
    const int ns = mv.ns, n = L.n, ldw = L.ldw;
    double *base = smem_int + (size_t)wib * L.per_warp;
    const int64_t gw = (int64_t)blockIdx.x * wpb + wib;          // global warp index
    double *mat = L.oMat >= 0 ? base + L.oMat : p.gmat + (size_t)gw * n * ldw;
    const Ctx c = make_ctx(base, mat, L);

    if (MODE != kModeIntegrate) {
        const int64_t i = gw;
        if (i >= p.n) return;
        for (int k = lane; k < ns; k += 32) c.y[1 + k] = p.Y[i * p.ldY + k];
        if (lane == 0) c.y[0] = p.T[i];
        __syncwarp();
        if (MODE == kModeRhs) {
            reactor_eval<false>(mv, iv, L, c, p.P[i], c.y, c.r, lane);
            for (int k = lane; k < n; k += 32) p.f[i * p.ldF + k] = c.r[k];
        } else {
            reactor_eval<true>(mv, iv, L, c, p.P[i], c.y, c.r, lane);
            double *Jo = p.J + (size_t)i * n * n;
            for (int r = 0; r < n; ++r)
                for (int col = lane; col < n; col += 32) Jo[(size_t)r * n + col] = c.A[r * ldw + col];
        }
        return;
    }

    const RosCoef &rc = p.rc;
    const int64_t ncell = p.n_dev ? *p.n_dev : p.n;
    for (;;) {
        int64_t i = 0;
        if (lane == 0) i = atomicAdd(p.queue, 1u);
        i = __shfl_sync(0xffffffffu, (long long)i, 0);
        if (i >= ncell) break;
        for (int k = lane; k < ns; k += 32) c.y[1 + k] = p.Y[i * p.ldY + k];
        if (lane == 0) c.y[0] = p.T[i];
        __syncwarp();
        const double Pi = p.P[i];
        const double T0 = c.y[0];
        const double Tign = T0 + p.ign_dT;
        const bool fixed = p.fixed_steps > 0;
        double t = 0.0, t_ign = -1.0;
        double h = fixed ? p.t_end / p.fixed_steps : (p.h0 > 0.0 ? p.h0 : p.t_end);
        bool first = true;
        int nacc = 0, nrej = 0, status = CHEM_CELL_OK;
        bool after_reject = false;
        while (t < p.t_end) {
            if ((int64_t)(nacc + nrej) >= p.max_steps) {
                status = CHEM_CELL_MAX_STEPS;
                break;
            }
            h = fmin(h, p.hmax);
            bool last = false;
            if (h >= (p.t_end - t) * (1.0 - 1e-10)) {     // reach t_end exactly
                h = p.t_end - t;
                last = true;
            }
            if (h < fmax(p.hmin, fmax(1e-290, 8.0 * 2.220446049250313e-16 * t))) {
                status = CHEM_CELL_STEP_UNDERFLOW;
                break;
            }
            // f(y) (the first stage's right-hand side, FP64) and the stage Jacobian
            if (p.jac32) {
                reactor_eval<false>(mv, iv, L, c, Pi, c.y, c.r, lane);
                reactor_jac_f32(mv, iv, L, c, Pi, c.y, lane);
            } else {
                reactor_eval<true>(mv, iv, L, c, Pi, c.y, c.r, lane);
            }
            if (first && p.h0 <= 0.0 && !fixed) {
                // starting step: 0.01 |y| / |f| in the weighted RMS norm (Hairer, Norsett &
                // Wanner, Solving ODEs I, Sec. II.4), at most the interval
                double a0 = 0.0, a1 = 0.0;
                for (int k = lane; k < n; k += 32) {
                    const double sc = p.atol + p.rtol * fabs(c.y[k]);
                    a0 += (c.y[k] / sc) * (c.y[k] / sc);
                    a1 += (c.r[k] / sc) * (c.r[k] / sc);
                }
                const double d0 = sqrt(warp_sum(a0) / n), d1 = sqrt(warp_sum(a1) / n);
                const double hs = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
                if (isfinite(hs) && hs < h) {
                    h = hs;
                    last = false;
                }
            }
            first = false;
            const double dg = 1.0 / (h * rc.gamma);
            for (int r = 0; r < n; ++r)
                for (int col = lane; col < n; col += 32) {
                    double *e = c.A + r * ldw + col;
                    *e = (r == col ? dg : 0.0) - *e;
                }
            __syncwarp();
            if (!lu_factor(c, n, ldw, lane)) {
                h *= 0.25;
                ++nrej;
                after_reject = true;
                continue;
            }
            for (int st = 0; st < kStages; ++st) {
                if (st > 0) {
                    for (int k = lane; k < n; k += 32) {
                        double v = c.y[k];
                        for (int jj = 0; jj < st; ++jj) v += rc.a[st][jj] * c.U[jj * L.nv + k];
                        c.ys[k] = v;
                    }
                    __syncwarp();
                    reactor_eval<false>(mv, iv, L, c, Pi, c.ys, c.r, lane);
                    const double ih = 1.0 / h;
                    for (int k = lane; k < n; k += 32) {
                        double v = c.r[k];
                        for (int jj = 0; jj < st; ++jj) v += rc.c[st][jj] * ih * c.U[jj * L.nv + k];
                        c.r[k] = v;
                    }
                    __syncwarp();
                }
                lu_solve(c, n, ldw, c.r, c.U + st * L.nv, lane);
            }
            double acc = 0.0;
            for (int k = lane; k < n; k += 32) {
                double yn = c.y[k], e = 0.0;
                for (int jj = 0; jj < kStages; ++jj) {
                    const double u = c.U[jj * L.nv + k];
                    yn += rc.m[jj] * u;
                    e += rc.e[jj] * u;
                }
                c.yn[k] = yn;
                const double sc = p.atol + p.rtol * fmax(fabs(c.y[k]), fabs(yn));
                const double z = e / sc;
                acc += z * z;
            }
            const double err = sqrt(warp_sum(acc) / (double)n);
            __syncwarp();
            if (fixed && !isfinite(err)) {
                status = CHEM_CELL_NONFINITE;
                break;
            }
            if (!fixed && !(err <= 1.0)) {
                const double fac = isfinite(err) ? fmax(0.2, 0.9 * pow(err, -1.0 / 3.0)) : 0.2;
                h *= fac;
                ++nrej;
                after_reject = true;
                continue;
            }
            const double Tn = c.yn[0], To = c.y[0];
            if (t_ign < 0.0 && Tn >= Tign && To < Tign)
                t_ign = t + h * (Tign - To) / (Tn - To);
            t = last ? p.t_end : t + h;
            for (int k = lane; k < n; k += 32) c.y[k] = c.yn[k];
            __syncwarp();
            ++nacc;
            double fac = err > 0.0 ? fmin(5.0, fmax(0.2, 0.9 * pow(err, -1.0 / 3.0))) : 5.0;
            if (after_reject) fac = fmin(fac, 1.0);
            after_reject = false;
            if (!fixed) h *= fac;
        }
        for (int k = lane; k < ns; k += 32) p.Yout[i * p.ldY + k] = c.y[1 + k];
        if (lane == 0) {
            p.Tout[i] = c.y[0];
            if (p.status) p.status[i] = status;
            if (p.nacc) p.nacc[i] = nacc;
            if (p.nrej) p.nrej[i] = nrej;
            if (p.t_ign) p.t_ign[i] = t_ign;
            if (status != CHEM_CELL_OK) atomicAdd(p.queue + 1, 1u);
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------

static constexpr size_t kSmemLimit = 227 * 1024;

struct LaunchShape {
    WarpLayout L;
    int wpb;             // warps per block
    size_t smem;
};

static chem_status shape_for(const chem_mech *m, LaunchShape *out)
{
    if (!m->vint.ok)
        return set_error(CHEM_EUNSUPPORTED,
                         "reactor kernels: a reaction has more than %d distinct species", kIntMax);
    WarpLayout Ls = make_layout(m->ns, true);
    size_t per = (size_t)Ls.per_warp * sizeof(double);
    if (per <= kSmemLimit) {
        int wpb = (int)(kSmemLimit / per);
        if (wpb > 8) wpb = 8;
        out->L = Ls;
        out->wpb = wpb;
        out->smem = per * wpb;
        return CHEM_OK;
    }
    WarpLayout Lg = make_layout(m->ns, false);
    per = (size_t)Lg.per_warp * sizeof(double);
    if (per > kSmemLimit)
        return set_error(CHEM_EUNSUPPORTED, "reactor kernels: %d species exceed shared memory",
                         m->ns);
    int wpb = (int)(kSmemLimit / per);
    if (wpb > 8) wpb = 8;
    out->L = Lg;
    out->wpb = wpb;
    out->smem = per * wpb;
    return CHEM_OK;
}

template <int MODE>
static SmemOptIn &smem_opt()
{
    static SmemOptIn opt;
    return opt;
}

static const RosCoef &coef()
{
    static const RosCoef r = make_coef();
    return r;
}

static chem_status common_checks(const chem_mech *m, int64_t n, const double *T, const double *P,
                                 const double *Y, int64_t ldY)
{
    if (!m) return set_error(CHEM_EINVAL, "mechanism is NULL");
    if (n < 0) return set_error(CHEM_EINVAL, "n_cells < 0");
    if (ldY < m->ns) return set_error(CHEM_EINVAL, "ldY below n_species=%d", m->ns);
    if (n > 0 && (!T || !P || !Y)) return set_error(CHEM_EINVAL, "NULL T, P or Y with n_cells > 0");
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != m->device) return set_error(CHEM_EINVAL, "mechanism lives on device %d", m->device);
    return CHEM_OK;
}

template <int MODE>
static chem_status launch_pointwise(const chem_mech *m, IntegParams &p, cudaStream_t s,
                                    const char *name)
{
    LaunchShape sh;
    chem_status st = shape_for(m, &sh);
    if (st != CHEM_OK) return st;
    p.L = sh.L;
    const int64_t blocks = (p.n + sh.wpb - 1) / sh.wpb;
    double *gmat = nullptr;
    if (MODE == kModeJac && sh.L.oMat < 0) {
        size_t bytes = (size_t)blocks * sh.wpb * sh.L.n * sh.L.ldw * sizeof(double);
        cudaError_t e = cudaMallocAsync((void **)&gmat, bytes, s);
        if (e != cudaSuccess) return set_error(CHEM_ENOMEM, "%s: workspace of %zu bytes: %s", name, bytes, cudaGetErrorString(e));
    }
    p.gmat = gmat;
    st = launch_opted(smem_opt<MODE>(), (const void *)k_reactor<MODE>, (int)kSmemLimit, name, [&] {
        k_reactor<MODE><<<(unsigned)blocks, sh.wpb * 32, sh.smem, s>>>(m->v64, m->vint, p);
    });
    if (st == CHEM_OK) g_launches.fetch_add(1);
    if (gmat) cudaFreeAsync(gmat, s);
    return st;
}

}  // namespace chem

using namespace chem;

extern "C" chem_status chem_ode_rhs(const chem_mech *m, int64_t n, const double *T, const double *P,
                                    const double *Y, int64_t ldY, double *f, int64_t ldF,
                                    void *stream)
{
    clear_error();
    chem_status st = common_checks(m, n, T, P, Y, ldY);
    if (st != CHEM_OK) return st;
    if (ldF < m->ns + 1) return set_error(CHEM_EINVAL, "ldF below n_species + 1");
    if (n > 0 && !f) return set_error(CHEM_EINVAL, "NULL f");
    if (n == 0) return CHEM_OK;
    IntegParams p;
    memset(&p, 0, sizeof p);
    p.n = n;
    p.T = T;
    p.P = P;
    p.Y = Y;
    p.ldY = ldY;
    p.f = f;
    p.ldF = ldF;
    return launch_pointwise<kModeRhs>(m, p, (cudaStream_t)stream, "ode_rhs");
}

extern "C" chem_status chem_ode_jacobian(const chem_mech *m, int64_t n, const double *T,
                                         const double *P, const double *Y, int64_t ldY, double *J,
                                         void *stream)
{
    clear_error();
    chem_status st = common_checks(m, n, T, P, Y, ldY);
    if (st != CHEM_OK) return st;
    if (n > 0 && !J) return set_error(CHEM_EINVAL, "NULL J");
    if (n == 0) return CHEM_OK;
    IntegParams p;
    memset(&p, 0, sizeof p);
    p.n = n;
    p.T = T;
    p.P = P;
    p.Y = Y;
    p.ldY = ldY;
    p.J = J;
    return launch_pointwise<kModeJac>(m, p, (cudaStream_t)stream, "ode_jacobian");
}

namespace chem {

static int64_t integrate_blocks(const LaunchShape &sh, int64_t n_max)
{
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_reactor<kModeIntegrate>, sh.wpb * 32, sh.smem);
    if (per_sm < 1) per_sm = 1;
    int64_t blocks = (int64_t)sm_limit(nsm) * per_sm;
    const int64_t need = (n_max + sh.wpb - 1) / sh.wpb;
    return blocks > need ? need : blocks;
}

static constexpr size_t kIntegHead = 256;   // cell queue and failure count

size_t integrate_header_bytes() { return kIntegHead; }

size_t integrate_workspace_bytes(const chem_mech *m, int64_t n_max)
{
    LaunchShape sh;
    if (!m || n_max < 1 || shape_for(m, &sh) != CHEM_OK) {
        clear_error();
        return 0;
    }
    const int64_t blocks = integrate_blocks(sh, n_max);
    const size_t mat = sh.L.oMat < 0 ? (size_t)blocks * sh.wpb * sh.L.n * sh.L.ldw * sizeof(double) : 0;
    return kIntegHead + mat;
}

// Enqueue one integration on `s`: clear the workspace header, launch the persistent kernel.
// No allocation and no synchronisation, so the two operations can be captured in a graph.
// With n_dev the kernel takes the cell count from device memory (at most n_max cells).
chem_status integrate_launch(const chem_mech *m, int64_t n_max, const int64_t *n_dev, double *T,
                             const double *P, double *Y, int64_t ldY, double t_end, double rtol,
                             double atol, const chem_integrate_opts *opts, int32_t *cell_status,
                             void *ws, size_t ws_bytes, cudaStream_t s)
{
    LaunchShape sh;
    chem_status st = shape_for(m, &sh);
    if (st != CHEM_OK) return st;
    const int64_t blocks = integrate_blocks(sh, n_max);
    const size_t mat = sh.L.oMat < 0 ? (size_t)blocks * sh.wpb * sh.L.n * sh.L.ldw * sizeof(double) : 0;
    if (!ws || ws_bytes < kIntegHead + mat)
        return set_error(CHEM_EINVAL, "integrate: workspace below %zu bytes", kIntegHead + mat);
    IntegParams p;
    memset(&p, 0, sizeof p);
    p.n = n_max;
    p.n_dev = n_dev;
    p.T = T;
    p.P = P;
    p.Y = Y;
    p.Tout = T;
    p.Yout = Y;
    p.ldY = ldY;
    p.t_end = t_end;
    p.rtol = rtol;
    p.atol = atol;
    p.h0 = (opts && opts->h_init > 0.0) ? opts->h_init : 0.0;
    p.hmin = (opts && opts->h_min > 0.0) ? opts->h_min : 0.0;
    p.hmax = (opts && opts->h_max > 0.0) ? opts->h_max : t_end;
    p.max_steps = (opts && opts->max_steps > 0) ? opts->max_steps : 100000;
    p.ign_dT = (opts && opts->ign_dT > 0.0) ? opts->ign_dT : 400.0;
    p.fixed_steps = (opts && opts->fixed_steps > 0) ? opts->fixed_steps : 0;
    p.jac32 = (opts && opts->jacobian_fp32) ? 1 : 0;
    p.t_ign = opts ? opts->t_ign : nullptr;
    p.nacc = opts ? opts->n_accepted : nullptr;
    p.nrej = opts ? opts->n_rejected : nullptr;
    p.status = cell_status;
    p.L = sh.L;
    p.rc = coef();
    p.queue = (unsigned int *)ws;
    p.gmat = mat ? (double *)((char *)ws + kIntegHead) : nullptr;
    cudaError_t e = cudaMemsetAsync(ws, 0, kIntegHead, s);
    if (e != cudaSuccess) return set_error(CHEM_ECUDA, "integrate: %s", cudaGetErrorString(e));
    st = launch_opted(smem_opt<kModeIntegrate>(), (const void *)k_reactor<kModeIntegrate>,
                      (int)kSmemLimit, "integrate", [&] {
                          k_reactor<kModeIntegrate><<<(unsigned)blocks, sh.wpb * 32, sh.smem, s>>>(
                              m->v64, m->vint, p);
                      });
    if (st == CHEM_OK) g_launches.fetch_add(1);
    return st;
}

chem_status integrate_checks(const chem_mech *m, int64_t n, const double *T, const double *P,
                             const double *Y, int64_t ldY, double t_end, double rtol, double atol)
{
    chem_status st = common_checks(m, n, T, P, Y, ldY);
    if (st != CHEM_OK) return st;
    if (!(t_end >= 0.0) || !isfinite(t_end)) return set_error(CHEM_EINVAL, "t_end must be finite, >= 0");
    if (!(rtol > 0.0) || !(atol >= 0.0)) return set_error(CHEM_EINVAL, "need rtol > 0 and atol >= 0");
    if (n >= (int64_t)1 << 31) return set_error(CHEM_EINVAL, "integrate: at most 2^31 - 1 cells per call");
    LaunchShape sh;
    return shape_for(m, &sh);
}

}  // namespace chem

extern "C" chem_status chem_integrate_cells(const chem_mech *m, int64_t n, double *T, const double *P,
                                            double *Y, int64_t ldY, double t_end, double rtol,
                                            double atol, const chem_integrate_opts *opts,
                                            int32_t *cell_status, void *stream)
{
    clear_error();
    chem_status st = integrate_checks(m, n, T, P, Y, ldY, t_end, rtol, atol);
    if (st != CHEM_OK) return st;
    if (n == 0) return CHEM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t wsb = integrate_workspace_bytes(m, n);
    void *ws = nullptr;
    cudaError_t e = cudaMallocAsync(&ws, wsb, s);
    if (e != cudaSuccess) return set_error(CHEM_ENOMEM, "integrate: workspace of %zu bytes: %s", wsb, cudaGetErrorString(e));
    unsigned int h_fail = 0;
    st = integrate_launch(m, n, nullptr, T, P, Y, ldY, t_end, rtol, atol, opts, cell_status, ws, wsb, s);
    if (st == CHEM_OK) {
        e = cudaMemcpyAsync(&h_fail, (unsigned int *)ws + 1, sizeof h_fail, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) st = set_error(CHEM_ECUDA, "integrate: %s", cudaGetErrorString(e));
    }
    cudaError_t e2 = cudaFreeAsync(ws, s);
    cudaError_t e3 = cudaStreamSynchronize(s);
    if (st != CHEM_OK) return st;
    if (e2 != cudaSuccess || e3 != cudaSuccess)
        return set_error(CHEM_ECUDA, "integrate: %s", cudaGetErrorString(e2 != cudaSuccess ? e2 : e3));
    if (h_fail) return set_error(CHEM_ENONCONV, "integrate: %u of %lld cells failed", h_fail, (long long)n);
    return CHEM_OK;
}

extern "C" chem_status chem_rosenbrock_tableau(int32_t *stages, double *gamma_ii, double *alpha,
                                               double *gamma, double *b, double *bhat)
{
    clear_error();
    if (stages) *stages = kStages;
    if (gamma_ii) *gamma_ii = kGammaII;
    for (int i = 0; i < 4; ++i) {
        for (int j = 0; j < 4; ++j) {
            if (alpha) alpha[i * 4 + j] = kAlpha[i][j];
            if (gamma) gamma[i * 4 + j] = kGammaIJ[i][j];
        }
        if (b) b[i] = kB[i];
        if (bhat) bhat[i] = kBhat[i];
    }
    return CHEM_OK;
}
