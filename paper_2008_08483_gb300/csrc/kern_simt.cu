// kern_simt.cu -- SIMT source-term kernels: FP64 and FP32 (double-float exponents).
//
// One thread per cell; all threads of a warp walk the reactions in the same order,
// so every per-reaction table load is a broadcast and every branch on the reaction
// kind is warp-uniform.  Per-cell species arrays live in shared memory laid out
// [species][thread] (conflict-free, each thread owns one column).
//
// Per reaction j (Eq. 4 in log space, Eqs. 5-11, Sec. 2.4):
//   ln q_f = sum_k nu'_kj ln C_k + ln k_inf,j + ln(third-body or falloff factor)
//   ln q_r = sum_k nu''_kj ln C_k + ln k_inf,j - ln K_c,j + (same factor)   [reversible]
//   omega_k += (nu''_kj - nu'_kj) (exp(ln q_f) - exp(ln q_r))
#include <math.h>
#include <string.h>

#include "chem_internal.h"

namespace chem {

// ---------------------------------------------------------------------------------------
// FP64
// ---------------------------------------------------------------------------------------

template <int BLK>
__global__ void __launch_bounds__(BLK)
k_source_f64(MechViewF64 mv, int64_t n, const double *__restrict__ T,
             const double *__restrict__ P, const double *__restrict__ Y, int64_t ldY,
             double *__restrict__ om, int64_t ldO)
{
    extern __shared__ double smem64[];
    const int ns = mv.ns, tid = threadIdx.x;
    const int64_t i = (int64_t)blockIdx.x * BLK + tid;
    if (i >= n) return;
    double *sC = smem64 + tid;                 // C_k        [k * BLK]
    double *sL = smem64 + ns * BLK + tid;      // ln C_k
    double *sW = smem64 + 2 * ns * BLK + tid;  // omega_k
    const double Ti = T[i], Pi = P[i];
    const double *Yi = Y + i * ldY;
    double sum = 0.0;
    for (int k = 0; k < ns; ++k) {
        double y = Yi[k];
        y = (y > 0.0 ? y : 0.0) * mv.invW[k];
        sC[k * BLK] = y;
        sum += y;
    }
    const double ctot = Pi / (kR * Ti);
    const double scale = sum > 0.0 ? ctot / sum : 0.0;
    for (int k = 0; k < ns; ++k) {
        double c = sC[k * BLK] * scale;
        sC[k * BLK] = c;
        sL[k * BLK] = log(c);                  // -inf for an absent species
        sW[k * BLK] = 0.0;
    }
    const double lnT = log(Ti), invT = 1.0 / Ti, tau = Ti * 1e-3;
    const int rg = Ti >= mv.t_mid ? 1 : 0;
    for (int j = 0; j < mv.nr; ++j) {
        const RxnF64 *R = mv.rxn + j;
        const double lkinf = R->lnA + R->b * lnT - R->EoR * invT;
        double lfac = 0.0;
        const int kind = R->kind;
        if (kind != 0) {
            double M = ctot;                   // sum_k eff_k C_k = c_tot + sum_k (eff_k - 1) C_k
            for (int t = R->tb_begin; t < R->tb_end; ++t) M += mv.tb_e[t] * sC[mv.tb_sp[t] * BLK];
            if (kind == 1) {
                lfac = log(M);
            } else {
                const double lk0 = R->low[0] + R->low[1] * lnT - R->low[2] * invT;
                const double Pr = exp(lk0 - lkinf) * M;
                if (Pr > 0.0) {
                    lfac = log(Pr / (1.0 + Pr));
                    if (kind == 3) {
                        double Fc = R->troe[0] * exp(-Ti * R->troe[2]) +
                                    R->troe[1] * exp(-Ti * R->troe[3]);
                        if (R->troe[4] > 0.0) Fc += exp(-R->troe[4] * invT);
                        const double lFc = log10(Fc);
                        const double c = -0.4 - 0.67 * lFc, nn = 0.75 - 1.27 * lFc;
                        const double x = log10(Pr) + c;
                        const double f1 = x / (nn - 0.14 * x);
                        lfac += lFc / (1.0 + f1 * f1) * 2.302585092994045684;
                    }
                } else {
                    lfac = -INFINITY;
                }
            }
        }
        const double *kc = R->kc[rg];
        const double lKc = kc[0] + kc[1] * lnT +
                           tau * (kc[2] + tau * (kc[3] + tau * (kc[4] + tau * kc[5]))) +
                           kc[6] * invT;
        double sf = lkinf + lfac, sr = lkinf + lfac - lKc;
        for (int t = 0; t < R->nf; ++t) sf += R->nuf[t] * sL[R->spf[t] * BLK];
        for (int t = 0; t < R->nr; ++t) sr += R->nur[t] * sL[R->spr[t] * BLK];
        const double qf = exp(sf);
        const double qr = R->rev ? exp(sr) : 0.0;
        const double qn = qf - qr;
        for (int t = 0; t < R->nf; ++t) sW[R->spf[t] * BLK] -= R->nuf[t] * qn;
        for (int t = 0; t < R->nr; ++t) sW[R->spr[t] * BLK] += R->nur[t] * qn;
    }
    double *oi = om + i * ldO;
    for (int k = 0; k < ns; ++k) oi[k] = sW[k * BLK];
}

// ---------------------------------------------------------------------------------------
// FP32 with double-float exponent assembly
// ---------------------------------------------------------------------------------------

struct df {
    float h, l;
};

__device__ __forceinline__ df mkdf(float h, float l) { df r; r.h = h; r.l = l; return r; }
__device__ __forceinline__ df mkdf(float2 v) { return mkdf(v.x, v.y); }

// error-free transformations (Knuth two-sum, Dekker fast two-sum, FMA two-product); the
// explicit _rn intrinsics keep the compiler from contracting them
__device__ __forceinline__ df two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return mkdf(s, e);
}
__device__ __forceinline__ df quick_two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    return mkdf(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ df df_add(df a, df b)
{
    df s = two_sum(a.h, b.h);
    return quick_two_sum(s.h, __fadd_rn(__fadd_rn(a.l, b.l), s.l));
}
__device__ __forceinline__ df df_add_f(df a, float b)
{
    df s = two_sum(a.h, b);
    return quick_two_sum(s.h, __fadd_rn(a.l, s.l));
}
__device__ __forceinline__ df df_mul(df a, df b)
{
    float p = __fmul_rn(a.h, b.h);
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, fmaf(a.l, b.h, e));
    return quick_two_sum(p, e);
}
__device__ __forceinline__ df df_mul_f(df a, float b)
{
    float p = __fmul_rn(a.h, b);
    float e = fmaf(a.h, b, -p);
    e = fmaf(a.l, b, e);
    return quick_two_sum(p, e);
}
__device__ __forceinline__ df df_from_double(double x)
{
    float h = (float)x;
    return mkdf(h, (float)(x - (double)h));
}
// 2^x for a double-float exponent
__device__ __forceinline__ float df_exp2(df x)
{
    return exp2f(x.h) * fmaf(x.l, 0.69314718055994531f, 1.0f);
}

constexpr float kLg2Floor = -1000.0f;        // log2 X of an absent species (2^x underflows to 0)

__device__ __forceinline__ float ann_act(float x, int act)
{
    return act ? (x > 0.0f ? x : expm1f(x)) : fmaxf(x, 0.0f);
}

// With ANN, ln K_c of every reversible reaction comes from the approximate network
// (Sec. 2.3, Eqs. 12-14) evaluated once per cell, instead of the Gibbs layer.
template <int BLK, bool ANN>
__global__ void __launch_bounds__(BLK)
k_source_f32(MechViewF32 mv, KcAnnView av, int64_t n, const float *__restrict__ T,
             const float *__restrict__ P, const float *__restrict__ Y, int64_t ldY,
             float *__restrict__ om, int64_t ldO)
{
    extern __shared__ float smem32[];
    const int ns = mv.ns, tid = threadIdx.x;
    const int64_t i = (int64_t)blockIdx.x * BLK + tid;
    if (i >= n) return;
    float *sE = smem32 + tid;                  // integer part of log2 X_k (exact)
    float *sF = smem32 + ns * BLK + tid;       // log2 of the mantissa of X_k, in [-1, 0)
    float *sGh = smem32 + 2 * ns * BLK + tid;  // -g_k/(RT) in log2 units, double-float
    float *sGl = smem32 + 3 * ns * BLK + tid;
    float *sWs = smem32 + 4 * ns * BLK + tid;  // omega_k, compensated sum
    float *sWc = smem32 + 5 * ns * BLK + tid;
    float *sH = smem32 + 6 * ns * BLK + tid;   // ANN: two layers of hidden units
    const float Tf = T[i], Pf = P[i];
    const float *Yi = Y + i * ldY;
    double sum = 0.0;
    for (int k = 0; k < ns; ++k) {
        float y = Yi[k];
        y = (y > 0.0f ? y : 0.0f) * mv.spec[k].invW;
        sF[k * BLK] = y;
        sum += (double)y;
    }
    const double inv_sum = sum > 0.0 ? 1.0 / sum : 0.0;
    // per-cell features in double precision, kept as double-float pairs
    const double Td = (double)Tf;
    const double lg2Td = log2(Td);
    const df lg2T = df_from_double(lg2Td);
    const df invT = df_from_double(1.0 / Td);
    const double taud = Td * 1e-3;
    df phi[7];                                 // [1, log2 T, tau, tau^2, tau^3, tau^4, 1/T]
    phi[0] = mkdf(1.0f, 0.0f);
    phi[1] = lg2T;
    phi[2] = df_from_double(taud);
    phi[3] = df_from_double(taud * taud);
    phi[4] = df_from_double(taud * taud * taud);
    phi[5] = df_from_double(taud * taud * taud * taud);
    phi[6] = invT;
    const df lgct = df_from_double(log2((double)Pf) - log2(kR) - lg2Td);    // log2 c_tot
    const df lgpRT = df_add(mkdf(mv.lg2_pref_R), mkdf(-lg2T.h, -lg2T.l));  // log2(p_ref/RT)
    const int rg = Tf >= mv.t_mid ? 1 : 0;
    for (int k = 0; k < ns; ++k) {
        const double X = (double)sF[k * BLK] * inv_sum;
        float e, f;
        if (X > 0x1p-150) {
            int ex;
            const double m = frexp(X, &ex);    // X = m 2^ex, m in [0.5, 1)
            e = (float)ex;
            f = log2f((float)m);
        } else {
            e = kLg2Floor;
            f = 0.0f;
        }
        sE[k * BLK] = e;
        sF[k * BLK] = f;
        if (!ANN) {
            const float2 *c = mv.spec[k].gl[rg];
            df g = mkdf(c[0]);
            for (int m = 1; m < 7; ++m) g = df_add(g, df_mul(mkdf(c[m]), phi[m]));
            sGh[k * BLK] = g.h;
            sGl[k * BLK] = g.l;
        }
        sWs[k * BLK] = 0.0f;
        sWc[k * BLK] = 0.0f;
    }
    int cur = 0;                               // ANN: layer buffer holding the last layer
    if (ANN) {
        const float x = (logf(Tf) - av.x_mean) * av.x_inv_std;
        for (int h = 0; h < av.nh; ++h) sH[h * BLK] = ann_act(fmaf(av.w_in[h], x, av.b_in[h]), av.act);
        for (int l = 0; l + 1 < av.nl; ++l) {
            const float *W = av.w_hid + (size_t)l * av.nh * av.nh;
            for (int o = 0; o < av.nh; ++o) {
                float a = av.b_hid[l * av.nh + o];
                for (int h = 0; h < av.nh; ++h)
                    a = fmaf(W[o * av.nh + h], sH[(cur * kAnnMaxHidden + h) * BLK], a);
                sH[((cur ^ 1) * kAnnMaxHidden + o) * BLK] = ann_act(a, av.act);
            }
            cur ^= 1;
        }
    }
    for (int j = 0; j < mv.nr; ++j) {
        const RxnF32 *R = mv.rxn + j;
        // Arrhenius layer, log2 k_inf (Eq. 6)
        df tf = df_add(df_add(mkdf(R->kf[0]), df_mul(mkdf(R->kf[1]), lg2T)),
                       df_mul(mkdf(R->kf[2]), invT));
        // third-body / falloff factor, log2 (Sec. 2.4)
        df fac = mkdf(0.0f, 0.0f);
        bool dead = false;
        const int kind = R->kind;
        if (kind != 0) {
            float s = 1.0f;                    // M / c_tot = 1 + sum_k (eff_k - 1) X_k
            for (int t = R->tb_begin; t < R->tb_end; ++t) {
                const int k = mv.tb_sp[t];
                s = fmaf(mv.tb_e[t], ldexpf(exp2f(sF[k * BLK]), (int)sE[k * BLK]), s);
            }
            if (!(s > 0.0f)) {
                dead = true;
            } else {
                const df lgM = df_add_f(lgct, log2f(s));
                if (kind == 1) {
                    fac = lgM;
                } else {
                    df t0 = df_add(df_add(mkdf(R->k0[0]), df_mul(mkdf(R->k0[1]), lg2T)),
                                   df_mul(mkdf(R->k0[2]), invT));
                    df lPr = df_add(df_add(t0, mkdf(-tf.h, -tf.l)), lgM);   // log2 Pr
                    // log2(Pr / (1 + Pr)) without cancellation on either side of Pr = 1
                    if (lPr.h < 0.0f)
                        fac = df_add_f(lPr, -log2f(1.0f + exp2f(lPr.h)));
                    else
                        fac = mkdf(-log2f(1.0f + exp2f(-lPr.h)), 0.0f);
                    if (kind == 3) {
                        const float Tn = Tf;
                        float Fc = R->troe[0] * expf(-Tn * R->troe[2]) +
                                   R->troe[1] * expf(-Tn * R->troe[3]);
                        if (R->troe[4] > 0.0f) Fc += expf(-R->troe[4] / Tn);
                        const float lFc = log10f(Fc);
                        const float c = -0.4f - 0.67f * lFc, nn = 0.75f - 1.27f * lFc;
                        const float x = (lPr.h + lPr.l) * 0.30102999566398120f + c;
                        const float f1 = x / (nn - 0.14f * x);
                        fac = df_add_f(fac, lFc / (1.0f + f1 * f1) * 3.3219280948873623f);
                    }
                }
            }
        }
        float qn = 0.0f;
        if (!dead) {
            // forward: tf + ord' log2 c_tot + sum nu' log2 X + factor
            float ei = 0.0f, fs = 0.0f;
            for (int t = 0; t < R->nf; ++t) {
                const int k = R->spf[t];
                const float nu = (float)R->nuf[t];
                ei = fmaf(nu, sE[k * BLK], ei);
                fs = fmaf(nu, sF[k * BLK], fs);
            }
            df xf = df_add(df_add(tf, df_mul_f(lgct, (float)R->ordf)), fac);
            xf = df_add_f(df_add_f(xf, ei), fs);
            qn = df_exp2(xf);
            if (R->rev) {
                df lkc;
                float er = 0.0f, fr = 0.0f;
                if (ANN) {
                    // ln K_c = y_mean + y_std (b + sum_h w_h a_h) (Eq. 14), in log2 units
                    const float *w = av.w_out + (size_t)j * av.nh;
                    float a = av.b_out[j];
                    for (int h = 0; h < av.nh; ++h)
                        a = fmaf(w[h], sH[(cur * kAnnMaxHidden + h) * BLK], a);
                    lkc = mkdf(fmaf(av.y_std[j], a, av.y_mean[j]) * 1.4426950408889634f, 0.0f);
                    for (int t = 0; t < R->nr; ++t) {
                        const int k = R->spr[t];
                        const float nu = (float)R->nur[t];
                        er = fmaf(nu, sE[k * BLK], er);
                        fr = fmaf(nu, sF[k * BLK], fr);
                    }
                } else {
                    // log2 K_c = sum_k nu_kj (-g_k/RT) + dnu log2(p_ref/RT) (Eqs. 8-9)
                    lkc = df_mul_f(lgpRT, (float)R->dnu);
                    for (int t = 0; t < R->nr; ++t) {
                        const int k = R->spr[t];
                        const float nu = (float)R->nur[t];
                        lkc = df_add(lkc, df_mul_f(mkdf(sGh[k * BLK], sGl[k * BLK]), nu));
                        er = fmaf(nu, sE[k * BLK], er);
                        fr = fmaf(nu, sF[k * BLK], fr);
                    }
                    for (int t = 0; t < R->nf; ++t) {
                        const int k = R->spf[t];
                        lkc = df_add(lkc, df_mul_f(mkdf(sGh[k * BLK], sGl[k * BLK]),
                                                   -(float)R->nuf[t]));
                    }
                }
                df xr = df_add(df_add(tf, df_mul_f(lgct, (float)R->ordr)), fac);
                xr = df_add(xr, mkdf(-lkc.h, -lkc.l));
                xr = df_add_f(df_add_f(xr, er), fr);
                qn -= df_exp2(xr);
            }
        }
        // omega_k += nu_kj q_net (Eq. 2), compensated accumulation
        for (int t = 0; t < R->nf; ++t) {
            const int k = R->spf[t];
            const df s = two_sum(sWs[k * BLK], -(float)R->nuf[t] * qn);
            sWs[k * BLK] = s.h;
            sWc[k * BLK] += s.l;
        }
        for (int t = 0; t < R->nr; ++t) {
            const int k = R->spr[t];
            const df s = two_sum(sWs[k * BLK], (float)R->nur[t] * qn);
            sWs[k * BLK] = s.h;
            sWc[k * BLK] += s.l;
        }
    }
    float *oi = om + i * ldO;
    for (int k = 0; k < ns; ++k) oi[k] = sWs[k * BLK] + sWc[k * BLK];
}

// ---------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------

constexpr size_t kMaxDynSmem = 227 * 1024;

// Opt a kernel in to the full dynamic shared memory once per device.
template <typename K>
static chem_status smem_opt_in(K kern, std::atomic<uint32_t> &done_mask, const char *name)
{
    int dev = 0;
    cudaGetDevice(&dev);
    const uint32_t bit = 1u << (dev & 31);
    if (done_mask.load() & bit) return CHEM_OK;
    cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxDynSmem);
    if (e != cudaSuccess) return set_error(CHEM_ECUDA, "%s: %s", name, cudaGetErrorString(e));
    done_mask.fetch_or(bit);
    return CHEM_OK;
}

template <int BLK, typename K, typename... A>
static chem_status launch_rows(K kern, std::atomic<uint32_t> &mask, size_t smem, int64_t n,
                               cudaStream_t s, const char *name, A... args)
{
    chem_status st = smem_opt_in(kern, mask, name);
    if (st != CHEM_OK) return st;
    kern<<<(unsigned)((n + BLK - 1) / BLK), BLK, smem, s>>>(args...);
    g_launches.fetch_add(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(CHEM_ECUDA, "%s launch: %s", name, cudaGetErrorString(e));
    return CHEM_OK;
}

chem_status launch_source_fp64(const chem_mech *m, int64_t n, const double *T, const double *P,
                               const double *Y, int64_t ldY, double *om, int64_t ldO,
                               cudaStream_t s)
{
    static std::atomic<uint32_t> m64{0}, m32{0};
    const size_t per = 3 * sizeof(double) * (size_t)m->ns;
    if (per * 64 <= 200 * 1024)
        return launch_rows<64>(k_source_f64<64>, m64, per * 64, n, s, "fp64", m->v64, n, T, P,
                               Y, ldY, om, ldO);
    if (per * 32 <= kMaxDynSmem)
        return launch_rows<32>(k_source_f64<32>, m32, per * 32, n, s, "fp64", m->v64, n, T, P,
                               Y, ldY, om, ldO);
    return set_error(CHEM_EUNSUPPORTED, "fp64: %d species exceed the SIMT kernel", m->ns);
}

chem_status launch_source_fp32(const chem_mech *m, int64_t n, const float *T, const float *P,
                               const float *Y, int64_t ldY, float *om, int64_t ldO,
                               cudaStream_t s)
{
    static std::atomic<uint32_t> m64{0}, m32{0};
    const size_t per = 6 * sizeof(float) * (size_t)m->ns;
    KcAnnView none;
    memset(&none, 0, sizeof none);
    if (per * 64 <= 200 * 1024)
        return launch_rows<64>(k_source_f32<64, false>, m64, per * 64, n, s, "fp32", m->v32,
                               none, n, T, P, Y, ldY, om, ldO);
    if (per * 32 <= kMaxDynSmem)
        return launch_rows<32>(k_source_f32<32, false>, m32, per * 32, n, s, "fp32", m->v32,
                               none, n, T, P, Y, ldY, om, ldO);
    return set_error(CHEM_EUNSUPPORTED, "fp32: %d species exceed the SIMT kernel", m->ns);
}

chem_status launch_source_fp32_ann(const chem_mech *m, const KcAnnView &av, int64_t n,
                                   const float *T, const float *P, const float *Y, int64_t ldY,
                                   float *om, int64_t ldO, cudaStream_t s)
{
    static std::atomic<uint32_t> m64{0}, m32{0};
    const size_t per = sizeof(float) * (6 * (size_t)m->ns + 2 * kAnnMaxHidden);
    if (per * 64 <= 200 * 1024)
        return launch_rows<64>(k_source_f32<64, true>, m64, per * 64, n, s, "fp32 ann", m->v32,
                               av, n, T, P, Y, ldY, om, ldO);
    if (per * 32 <= kMaxDynSmem)
        return launch_rows<32>(k_source_f32<32, true>, m32, per * 32, n, s, "fp32 ann", m->v32,
                               av, n, T, P, Y, ldY, om, ldO);
    return set_error(CHEM_EUNSUPPORTED, "fp32 ann: %d species exceed the SIMT kernel", m->ns);
}

// Exact ln K_c of every reaction (Eqs. 8-11, the FP64 folded Gibbs layer), one thread per
// cell: lnkc[i * ldK + j].
__global__ void k_log_kc(MechViewF64 mv, int64_t n, const double *__restrict__ T,
                         double *__restrict__ lnkc, int64_t ldK)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double Ti = T[i], lnT = log(Ti), invT = 1.0 / Ti, tau = Ti * 1e-3;
    const int rg = Ti >= mv.t_mid ? 1 : 0;
    for (int j = 0; j < mv.nr; ++j) {
        const double *kc = mv.rxn[j].kc[rg];
        lnkc[i * ldK + j] = kc[0] + kc[1] * lnT +
                            tau * (kc[2] + tau * (kc[3] + tau * (kc[4] + tau * kc[5]))) +
                            kc[6] * invT;
    }
}

chem_status launch_log_kc(const chem_mech *m, int64_t n, const double *T, double *lnkc,
                          int64_t ldK, cudaStream_t s)
{
    k_log_kc<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(m->v64, n, T, lnkc, ldK);
    g_launches.fetch_add(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(CHEM_ECUDA, "log_kc launch: %s", cudaGetErrorString(e));
    return CHEM_OK;
}

}  // namespace chem
