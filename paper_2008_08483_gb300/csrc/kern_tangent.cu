// kern_tangent.cu -- derivatives of omega with respect to (ln C, T): jvp and vjp one warp per
// cell, the dense Jacobian one thread per cell (SIMT, double or float).
//
// With q_f = k_f prod C^nu' and q_r = k_f / K_c prod C^nu'' (Eqs. 3, 7), per reaction
//   d ln q_f = sum_m nu'_m d ln C_m + d ln k_f
//   d ln q_r = sum_m nu''_m d ln C_m + d ln k_f - d ln K_c
//   d ln k_f = (b/T + (E/R)/T^2) dT + d ln(modifier)                             (Eq. 5)
//   d ln K_c / dT from the folded Gibbs polynomial (Eqs. 9-11)
//   modifier: third body M = sum_m eff_m C_m, d ln M = sum_m eff_m C_m d ln C_m / M;
//             falloff Pr / (1 + Pr) F(T, Pr), Pr = k0 M / k_inf, through the chain rule
//   d omega_k = sum_j nu_kj (q_f d ln q_f - q_r d ln q_r)                        (Eq. 2)
// sum_m eff_m C_m x_m is evaluated as sum_m C_m x_m + sum_{listed m} (eff_m - 1) C_m x_m.
#include <math.h>

#include <algorithm>
#include <string.h>

#include "chem_internal.h"
#include "rxn_terms.cuh"

namespace chem {

enum TangentMode { kJvp = 0, kVjp = 1, kJac = 2 };

template <typename R>
struct TanArgs {
    int64_t n;
    const R *T, *lnC;
    int64_t ldC;
    const R *dT, *dlnC;      // jvp tangent (dlnC row stride ldC)
    R *om;                   // jvp: omega (may be NULL)
    R *dom;                  // jvp: d omega
    int64_t ldO;
    const R *gw;             // vjp: cotangent of omega (row stride ldO)
    R *gT, *glnC;            // vjp outputs (glnC row stride ldC)
    R *J;                    // jac: [(k (ns + 1) + m) ldJ + i], m = ns is T
    int64_t ldJ;
};


template <typename R, int MODE, int BLK>
__global__ void __launch_bounds__(BLK) k_tangent(MechViewF64 mv, TanArgs<R> a)
{
    extern __shared__ unsigned char smem_tan[];
    R *sm = (R *)smem_tan;
    const int ns = mv.ns, tid = threadIdx.x;
    const int64_t i = (int64_t)blockIdx.x * BLK + tid;
    if (i >= a.n) return;
    R *sC = sm + tid;                           // C_m
    R *sL = sm + ns * BLK + tid;                // ln C_m
    R *sA = sm + 2 * ns * BLK + tid;            // jvp: d ln C_m; vjp: cotangent of omega_k
    R *sB = sm + 3 * ns * BLK + tid;            // jvp: d omega_k; vjp: g ln C_m; jac: V_k
    R *sW = sm + 4 * ns * BLK + tid;            // jvp: omega_k
    const R Ti = a.T[i];
    R ctot = 0, sdl = 0;
    for (int m = 0; m < ns; ++m) {
        const R l = a.lnC[i * a.ldC + m];
        const R c = rt_exp(l);
        sL[m * BLK] = l;
        sC[m * BLK] = c;
        ctot += c;
        if (MODE == kJvp) {
            const R d = a.dlnC[i * a.ldC + m];
            sA[m * BLK] = d;
            sdl += c * d;
            sB[m * BLK] = 0;
            sW[m * BLK] = 0;
        } else if (MODE == kVjp) {
            sA[m * BLK] = a.gw[i * a.ldO + m];
            sB[m * BLK] = 0;
        } else {
            sB[m * BLK] = 0;
            for (int mm = 0; mm <= ns; ++mm) a.J[((int64_t)m * (ns + 1) + mm) * a.ldJ + i] = 0;
        }
    }
    const R dT = MODE == kJvp ? a.dT[i] : R(0);
    const TFeat<R> tfe = t_features<R>(Ti, mv.t_mid);
    R gT = 0, Wtb = 0;      // vjp: cotangent of T; weight of the c_tot part of M
    for (int j = 0; j < mv.nr; ++j) {
        const RxnF64 *X = mv.rxn + j;
        const int kind = X->kind;
        R M = 1;
        if (kind != 0) {
            M = ctot;
            for (int t = X->tb_begin; t < X->tb_end; ++t) M += R(mv.tb_e[t]) * sC[mv.tb_sp[t] * BLK];
        }
        const RxnTerms<R> rt = rxn_terms<R>(X, tfe, M);
        if (rt.dead) continue;
        const R lkinf = rt.lkinf, lmod = rt.lmod, dmod_dlM = rt.dmod_dlM, dmod_dT = rt.dmod_dT;
        const R lKc = rt.lKc, dlKc = rt.dlKc, dlkinf = rt.dlkinf;
        R sf = lkinf + lmod, sr = lkinf + lmod - lKc;
        for (int t = 0; t < X->nf; ++t) sf += R(X->nuf[t]) * sL[X->spf[t] * BLK];
        for (int t = 0; t < X->nr; ++t) sr += R(X->nur[t]) * sL[X->spr[t] * BLK];
        const R qf = rt_exp(sf);
        const R qr = X->rev ? rt_exp(sr) : R(0);
        const R dlkf_dT = dlkinf + dmod_dT;            // d ln k_f / dT
        if (MODE == kJvp) {
            R dlM = 0;
            if (kind != 0) {
                R s = sdl;
                for (int t = X->tb_begin; t < X->tb_end; ++t) {
                    const int m = mv.tb_sp[t];
                    s += R(mv.tb_e[t]) * sC[m * BLK] * sA[m * BLK];
                }
                dlM = s / M;
            }
            R tf = dlkf_dT * dT + dmod_dlM * dlM, tr = (dlkf_dT - dlKc) * dT + dmod_dlM * dlM;
            for (int t = 0; t < X->nf; ++t) tf += R(X->nuf[t]) * sA[X->spf[t] * BLK];
            for (int t = 0; t < X->nr; ++t) tr += R(X->nur[t]) * sA[X->spr[t] * BLK];
            const R qn = qf - qr, dqn = qf * tf - qr * tr;
            for (int t = 0; t < X->nf; ++t) {
                sB[X->spf[t] * BLK] -= R(X->nuf[t]) * dqn;
                sW[X->spf[t] * BLK] -= R(X->nuf[t]) * qn;
            }
            for (int t = 0; t < X->nr; ++t) {
                sB[X->spr[t] * BLK] += R(X->nur[t]) * dqn;
                sW[X->spr[t] * BLK] += R(X->nur[t]) * qn;
            }
        } else if (MODE == kVjp) {
            R aa = 0;                                  // sum_k nu_kj g omega_k
            for (int t = 0; t < X->nf; ++t) aa -= R(X->nuf[t]) * sA[X->spf[t] * BLK];
            for (int t = 0; t < X->nr; ++t) aa += R(X->nur[t]) * sA[X->spr[t] * BLK];
            const R uf = aa * qf, ur = aa * qr;
            for (int t = 0; t < X->nf; ++t) sB[X->spf[t] * BLK] += uf * R(X->nuf[t]);
            for (int t = 0; t < X->nr; ++t) sB[X->spr[t] * BLK] -= ur * R(X->nur[t]);
            gT += uf * dlkf_dT - ur * (dlkf_dT - dlKc);
            if (kind != 0) {
                const R w = (uf - ur) * dmod_dlM / M;  // times eff_m C_m for every m
                Wtb += w;
                for (int t = X->tb_begin; t < X->tb_end; ++t) {
                    const int m = mv.tb_sp[t];
                    sB[m * BLK] += w * R(mv.tb_e[t]) * sC[m * BLK];
                }
            }
        } else {
            // d omega_k / d ln C_m and d omega_k / dT for the species of this reaction
            const R dqT = qf * dlkf_dT - qr * (dlkf_dT - dlKc);
            const R w = kind != 0 ? (qf - qr) * dmod_dlM / M : R(0);
            auto row = [&](int k, R nu) {
                R *Jk = a.J + (int64_t)k * (ns + 1) * a.ldJ + i;
                Jk[(int64_t)ns * a.ldJ] += nu * dqT;
                for (int t = 0; t < X->nf; ++t)
                    Jk[(int64_t)X->spf[t] * a.ldJ] += nu * qf * R(X->nuf[t]);
                for (int t = 0; t < X->nr; ++t)
                    Jk[(int64_t)X->spr[t] * a.ldJ] -= nu * qr * R(X->nur[t]);
                if (kind != 0) {
                    sB[k * BLK] += nu * w;                // c_tot part: C_m V_k at the end
                    for (int t = X->tb_begin; t < X->tb_end; ++t) {
                        const int m = mv.tb_sp[t];
                        Jk[(int64_t)m * a.ldJ] += nu * w * R(mv.tb_e[t]) * sC[m * BLK];
                    }
                }
            };
            for (int t = 0; t < X->nf; ++t) row(X->spf[t], -R(X->nuf[t]));
            for (int t = 0; t < X->nr; ++t) row(X->spr[t], R(X->nur[t]));
        }
    }
    if (MODE == kJvp) {
        for (int k = 0; k < ns; ++k) {
            a.dom[i * a.ldO + k] = sB[k * BLK];
            if (a.om) a.om[i * a.ldO + k] = sW[k * BLK];
        }
    } else if (MODE == kVjp) {
        a.gT[i] = gT;
        for (int m = 0; m < ns; ++m) a.glnC[i * a.ldC + m] = sB[m * BLK] + Wtb * sC[m * BLK];
    } else {
        for (int k = 0; k < ns; ++k) {
            const R v = sB[k * BLK];
            if (v == R(0)) continue;
            R *Jk = a.J + (int64_t)k * (ns + 1) * a.ldJ + i;
            for (int m = 0; m < ns; ++m) Jk[(int64_t)m * a.ldJ] += v * sC[m * BLK];
        }
    }
}


// ---------------------------------------------------------------------------------------
// Warp-per-cell jvp and vjp.  One warp per cell: the lanes take the species (C = exp ln C
// and the tangent or cotangent rows, coalesced), then the reactions (one slot of the
// kind-grouped order per lane: the rate terms, q_f, q_r and the reaction's tangent scalars,
// written to per-reaction arrays in shared memory), then the species again, gathering from
// the species-major lists in a fixed order (no atomics: results do not depend on the
// launch).  The per-cell arithmetic is that of k_tangent above.
// ---------------------------------------------------------------------------------------
constexpr int kTanWarps = 8;           // warps per block, at most

template <typename R>
__device__ __forceinline__ R tw_sum(R v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename R, int MODE>
__global__ void __launch_bounds__(32 * kTanWarps) k_tangent_w(MechViewF64 mv, IntView iv, TanArgs<R> a)
{
    extern __shared__ unsigned char smem_tw[];
    const int ns = mv.ns, nr = mv.nr, lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    if (i >= a.n) return;
    R *sC = (R *)smem_tw + (size_t)wib * (3 * ns + 3 * nr);
    R *sL = sC + ns;               // ln C_m
    R *sA = sL + ns;               // jvp: d ln C_m; vjp: cotangent of omega_k
    R *sP = sA + ns;               // jvp: q_net,j; vjp: u_j q_f,j
    R *sQ = sP + nr;               // jvp: d q_net,j; vjp: u_j q_r,j
    R *sV = sQ + nr;               // vjp: (u_j q_net,j) d ln mod / d ln M / M (third body)
    const R Ti = a.T[i];
    R ctot = 0, sdl = 0;
    for (int m = lane; m < ns; m += 32) {
        const R l = a.lnC[i * a.ldC + m];
        const R c = rt_exp(l);
        sL[m] = l;
        sC[m] = c;
        ctot += c;
        if (MODE == kJvp) {
            const R d = a.dlnC[i * a.ldC + m];
            sA[m] = d;
            sdl += c * d;
        } else {
            sA[m] = a.gw[i * a.ldO + m];
        }
    }
    ctot = tw_sum(ctot);
    if (MODE == kJvp) sdl = tw_sum(sdl);
    const R dT = MODE == kJvp ? a.dT[i] : R(0);
    const TFeat<R> tfe = t_features<R>(Ti, mv.t_mid);
    __syncwarp();
    R gT = 0, Wtb = 0;
    for (int sl = lane; sl < iv.n_slots; sl += 32) {
        const int j = iv.order[sl];
        if (j < 0) continue;
        const RxnF64 *X = mv.rxn + j;
        const int kind = X->kind;
        R M = 1;
        if (kind != 0) {
            M = ctot;
            for (int t = X->tb_begin; t < X->tb_end; ++t) M += R(mv.tb_e[t]) * sC[mv.tb_sp[t]];
        }
        const RxnTerms<R> rt = rxn_terms<R>(X, tfe, M);
        if (rt.dead) {
            sP[j] = 0;
            sQ[j] = 0;
            if (MODE == kVjp) sV[j] = 0;
            continue;
        }
        R sf = rt.lkinf + rt.lmod, sr = rt.lkinf + rt.lmod - rt.lKc;
        for (int t = 0; t < X->nf; ++t) sf += R(X->nuf[t]) * sL[X->spf[t]];
        for (int t = 0; t < X->nr; ++t) sr += R(X->nur[t]) * sL[X->spr[t]];
        const R qf = rt_exp(sf);
        const R qr = X->rev ? rt_exp(sr) : R(0);
        const R dlkf_dT = rt.dlkinf + rt.dmod_dT;
        if (MODE == kJvp) {
            R dlM = 0;
            if (kind != 0) {
                R s = sdl;
                for (int t = X->tb_begin; t < X->tb_end; ++t) {
                    const int m = mv.tb_sp[t];
                    s += R(mv.tb_e[t]) * sC[m] * sA[m];
                }
                dlM = s / M;
            }
            R tf = dlkf_dT * dT + rt.dmod_dlM * dlM, tr = (dlkf_dT - rt.dlKc) * dT + rt.dmod_dlM * dlM;
            for (int t = 0; t < X->nf; ++t) tf += R(X->nuf[t]) * sA[X->spf[t]];
            for (int t = 0; t < X->nr; ++t) tr += R(X->nur[t]) * sA[X->spr[t]];
            sP[j] = qf - qr;
            sQ[j] = qf * tf - qr * tr;
        } else {
            R aa = 0;                              // sum_k nu_kj g omega_k
            for (int t = 0; t < X->nf; ++t) aa -= R(X->nuf[t]) * sA[X->spf[t]];
            for (int t = 0; t < X->nr; ++t) aa += R(X->nur[t]) * sA[X->spr[t]];
            const R uf = aa * qf, ur = aa * qr;
            sP[j] = uf;
            sQ[j] = ur;
            gT += uf * dlkf_dT - ur * (dlkf_dT - rt.dlKc);
            R w = 0;
            if (kind != 0) {
                w = (uf - ur) * rt.dmod_dlM / M;   // times eff_m C_m for every m
                Wtb += w;
            }
            sV[j] = w;
        }
    }
    if (MODE == kVjp) {
        gT = tw_sum(gT);
        Wtb = tw_sum(Wtb);
    }
    __syncwarp();
    for (int e = mv.lane_ptr[lane]; e < mv.lane_ptr[lane + 1]; ++e) {
        const int k = mv.lane_sp[e];
        if (MODE == kJvp) {
            // d omega_k = sum_j nu_kj d q_net,j and omega_k, in the species-major order
            R d = 0, w = 0;
            for (int q = mv.col_ptr[k]; q < mv.col_ptr[k + 1]; ++q) {
                const int j = mv.col_rxn[q];
                const R nu = R(mv.col_nu[q]);
                d += nu * sQ[j];
                w += nu * sP[j];
            }
            a.dom[i * a.ldO + k] = d;
            if (a.om) a.om[i * a.ldO + k] = w;
        } else {
            // g ln C_m = sum_j (nu'_mj u q_f - nu''_mj u q_r) + C_m (sum_j w_j (1 + listed
            // eff_mj - 1))
            R g = 0, t = 0;
            for (int q = mv.sd_ptr[k]; q < mv.sd_ptr[k + 1]; ++q) {
                const int j = mv.sd_rxn[q];
                g += R(mv.sd_nuf[q]) * sP[j] - R(mv.sd_nur[q]) * sQ[j];
            }
            for (int q = mv.ts_ptr[k]; q < mv.ts_ptr[k + 1]; ++q) t += R(mv.ts_e[q]) * sV[mv.ts_rxn[q]];
            a.glnC[i * a.ldC + k] = g + (t + Wtb) * sC[k];
        }
    }
    if (MODE == kVjp && lane == 0) a.gT[i] = gT;
}

template <typename R, int MODE>
static chem_status launch_tan(const chem_mech *m, const TanArgs<R> &a, cudaStream_t s,
                              const char *name)
{
    static SmemOptIn done64, done32;
    const size_t per = 5 * sizeof(R) * (size_t)m->ns;
    auto go = [&](auto kern, int blk, SmemOptIn &done) -> chem_status {
        chem_status st = launch_opted(done, (const void *)kern, 227 * 1024, name, [&] {
            kern<<<(unsigned)((a.n + blk - 1) / blk), blk, per * blk, s>>>(m->v64, a);
        });
        if (st == CHEM_OK) g_launches.fetch_add(1);
        return st;
    };
    if (per * 64 <= 200 * 1024) return go(k_tangent<R, MODE, 64>, 64, done64);
    if (per * 32 <= 227 * 1024) return go(k_tangent<R, MODE, 32>, 32, done32);
    return set_error(CHEM_EUNSUPPORTED, "%s: %d species exceed the SIMT kernel", name, m->ns);
}

// Warp-per-cell launch; false in *used when the per-warp arrays do not fit in shared memory.
template <typename R, int MODE>
static chem_status launch_tan_w(const chem_mech *m, const TanArgs<R> &a, cudaStream_t s,
                                const char *name, bool *used)
{
    static SmemOptIn done;
    const size_t per = sizeof(R) * (3 * (size_t)m->ns + 3 * (size_t)m->nr);
    const int wpb = (int)std::min<size_t>((size_t)kTanWarps, (size_t)(227 * 1024) / per);
    *used = wpb >= 1;
    if (!*used) return CHEM_OK;
    const int64_t blocks = (a.n + wpb - 1) / wpb;
    chem_status st = launch_opted(done, (const void *)k_tangent_w<R, MODE>, 227 * 1024, name, [&] {
        k_tangent_w<R, MODE><<<(unsigned)blocks, 32 * wpb, per * wpb, s>>>(m->v64, m->vint, a);
    });
    if (st == CHEM_OK) g_launches.fetch_add(1);
    return st;
}

// jvp and vjp take the warp-per-cell kernel (it needs the kind-grouped reaction order, built
// when every reaction has at most kIntMax species, and its per-warp arrays in shared memory);
// the dense Jacobian, and mechanisms beyond those limits, the thread-per-cell one.
template <typename R>
chem_status tangent_dispatch(const chem_mech *m, int mode, const TanArgs<R> &a, cudaStream_t s)
{
    bool used = false;
    chem_status st = CHEM_OK;
    switch (mode) {
    case kJvp:
        if (m->vint.ok) st = launch_tan_w<R, kJvp>(m, a, s, "jvp", &used);
        return used ? st : launch_tan<R, kJvp>(m, a, s, "jvp");
    case kVjp:
        if (m->vint.ok) st = launch_tan_w<R, kVjp>(m, a, s, "vjp", &used);
        return used ? st : launch_tan<R, kVjp>(m, a, s, "vjp");
    default: return launch_tan<R, kJac>(m, a, s, "jacobian");
    }
}

}  // namespace chem

using namespace chem;

static chem_status tan_common(const chem_mech *m, int64_t n, const void *T, const void *lnC,
                              int64_t ldC, chem_precision prec)
{
    if (!m) return set_error(CHEM_EINVAL, "mechanism is NULL");
    if (n < 0) return set_error(CHEM_EINVAL, "n_cells < 0");
    if (ldC < m->ns) return set_error(CHEM_EINVAL, "ldC below n_species=%d", m->ns);
    if (prec != CHEM_FP64 && prec != CHEM_FP32)
        return set_error(CHEM_EUNSUPPORTED, "derivatives are built for CHEM_FP64 and CHEM_FP32");
    if (n > 0 && (!T || !lnC)) return set_error(CHEM_EINVAL, "NULL T or lnC with n_cells > 0");
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != m->device) return set_error(CHEM_EINVAL, "mechanism lives on device %d", m->device);
    return CHEM_OK;
}

template <typename R>
static TanArgs<R> targs(int64_t n, const void *T, const void *lnC, int64_t ldC)
{
    TanArgs<R> a;
    memset(&a, 0, sizeof a);
    a.n = n;
    a.T = (const R *)T;
    a.lnC = (const R *)lnC;
    a.ldC = ldC;
    return a;
}

extern "C" chem_status chem_source_term_jvp(const chem_mech *m, int64_t n, const void *T,
                                            const void *lnC, int64_t ldC, const void *dT,
                                            const void *dlnC, void *omega, void *domega,
                                            int64_t ldO, chem_precision prec, void *stream)
{
    clear_error();
    chem_status st = tan_common(m, n, T, lnC, ldC, prec);
    if (st != CHEM_OK) return st;
    if (ldO < m->ns) return set_error(CHEM_EINVAL, "ldO below n_species=%d", m->ns);
    if (n == 0) return CHEM_OK;
    if (!dT || !dlnC || !domega) return set_error(CHEM_EINVAL, "NULL tangent or output");
    cudaStream_t s = (cudaStream_t)stream;
    if (prec == CHEM_FP64) {
        TanArgs<double> a = targs<double>(n, T, lnC, ldC);
        a.dT = (const double *)dT;
        a.dlnC = (const double *)dlnC;
        a.om = (double *)omega;
        a.dom = (double *)domega;
        a.ldO = ldO;
        return tangent_dispatch<double>(m, kJvp, a, s);
    }
    TanArgs<float> a = targs<float>(n, T, lnC, ldC);
    a.dT = (const float *)dT;
    a.dlnC = (const float *)dlnC;
    a.om = (float *)omega;
    a.dom = (float *)domega;
    a.ldO = ldO;
    return tangent_dispatch<float>(m, kJvp, a, s);
}

extern "C" chem_status chem_source_term_vjp(const chem_mech *m, int64_t n, const void *T,
                                            const void *lnC, int64_t ldC, const void *g_omega,
                                            int64_t ldG, void *g_T, void *g_lnC,
                                            chem_precision prec, void *stream)
{
    clear_error();
    chem_status st = tan_common(m, n, T, lnC, ldC, prec);
    if (st != CHEM_OK) return st;
    if (ldG < m->ns) return set_error(CHEM_EINVAL, "ldG below n_species=%d", m->ns);
    if (n == 0) return CHEM_OK;
    if (!g_omega || !g_T || !g_lnC) return set_error(CHEM_EINVAL, "NULL cotangent or output");
    cudaStream_t s = (cudaStream_t)stream;
    if (prec == CHEM_FP64) {
        TanArgs<double> a = targs<double>(n, T, lnC, ldC);
        a.gw = (const double *)g_omega;
        a.ldO = ldG;
        a.gT = (double *)g_T;
        a.glnC = (double *)g_lnC;
        return tangent_dispatch<double>(m, kVjp, a, s);
    }
    TanArgs<float> a = targs<float>(n, T, lnC, ldC);
    a.gw = (const float *)g_omega;
    a.ldO = ldG;
    a.gT = (float *)g_T;
    a.glnC = (float *)g_lnC;
    return tangent_dispatch<float>(m, kVjp, a, s);
}

extern "C" chem_status chem_source_term_jacobian(const chem_mech *m, int64_t n, const void *T,
                                                 const void *lnC, int64_t ldC, void *J,
                                                 int64_t ldJ, chem_precision prec, void *stream)
{
    clear_error();
    chem_status st = tan_common(m, n, T, lnC, ldC, prec);
    if (st != CHEM_OK) return st;
    if (ldJ < n) return set_error(CHEM_EINVAL, "ldJ below n_cells");
    if (n == 0) return CHEM_OK;
    if (!J) return set_error(CHEM_EINVAL, "NULL Jacobian");
    cudaStream_t s = (cudaStream_t)stream;
    if (prec == CHEM_FP64) {
        TanArgs<double> a = targs<double>(n, T, lnC, ldC);
        a.J = (double *)J;
        a.ldJ = ldJ;
        return tangent_dispatch<double>(m, kJac, a, s);
    }
    TanArgs<float> a = targs<float>(n, T, lnC, ldC);
    a.J = (float *)J;
    a.ldJ = ldJ;
    return tangent_dispatch<float>(m, kJac, a, s);
}
