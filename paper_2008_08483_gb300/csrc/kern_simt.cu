// kern_simt.cu -- SIMT source-term kernels: FP64 and FP32 (double-float exponents).
//
// Both take one warp per cell (several consecutive cells per warp for large batches): the
// lanes take the cell's species, then its reactions (one slot of the kind-grouped order per
// lane, so kind branches are warp-uniform and record fields load coalesced from slot-major
// word tables), then omega by species (a gather over the species-major net stoichiometry,
// so results do not depend on an atomic order).
//
// Per reaction j (Eq. 4 in log space, Eqs. 5-11, Sec. 2.4):
//   ln q_f = sum_k nu'_kj ln C_k + ln k_inf,j + ln(third-body or falloff factor)
//   ln q_r = sum_k nu''_kj ln C_k + ln k_inf,j - ln K_c,j + (same factor)   [reversible]
//   omega_k += (nu''_kj - nu'_kj) (exp(ln q_f) - exp(ln q_r))
#include <math.h>
#include <stddef.h>
#include <string.h>

#include "chem_internal.h"

namespace chem {

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

// One warp per cell, cpw (1..32) consecutive cells per warp: 32 once the batch fills the GPU,
// fewer for small batches so that every resident warp gets work.  A first pass with one lane
// per cell computes the per-cell features (FP64, converted to double-float pairs) of the
// warp's cells; then for
// each cell the lanes take its species (z_k = Y_k / W_k from one coalesced row, log2 z_k as
// an exact exponent and the log2 of the mantissa, the Gibbs layer, sum_k z_k by a warp
// reduction), then its reactions (lane = reaction slot, slots grouped by kind so that the
// kind branches are warp-uniform), then omega by species (a gather over the species-major
// net stoichiometry, compensated, one coalesced row store).  With ANN, ln K_c of every
// reversible reaction comes from the approximate network (Sec. 2.3, Eqs. 12-14), whose hidden
// units the lanes evaluate once per cell, instead of the Gibbs layer.
constexpr int kF32Warps = 8;                   // warps per block
constexpr int kCellScalars = 16;               // per-cell scalars kept in shared memory

__device__ __forceinline__ df df_warp_sum(df v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const df o = mkdf(__shfl_xor_sync(0xffffffffu, v.h, off),
                          __shfl_xor_sync(0xffffffffu, v.l, off));
        v = df_add(v, o);
    }
    return v;
}

// log2 of a positive double-float: exact exponent + log2 of the mantissa + the low part
__device__ __forceinline__ df df_log2(df x)
{
    int ex;
    const float m = frexpf(x.h, &ex);          // x.h = m 2^ex, m in [0.5, 1)
    return df_add_f(two_sum((float)ex, log2f(m)), x.l / x.h * 1.4426950408889634f);
}

// One reaction record read from the slot-major word table: 32 lanes loading one field of 32
// consecutive slots make one coalesced load.
struct RxnW {
    const uint32_t *p;                         // word 0 of this slot
    int stride;                                // slots per word row
    __device__ __forceinline__ uint32_t word(size_t b) const { return __ldg(p + (b / 4) * (size_t)stride); }
    __device__ __forceinline__ float f(size_t b) const { return __uint_as_float(word(b)); }
    __device__ __forceinline__ int i(size_t b) const { return (int)word(b); }
    __device__ __forceinline__ df d2(size_t b) const { return mkdf(f(b), f(b + 4)); }
    __device__ __forceinline__ double dbl(size_t b) const
    {
        return __hiloint2double((int)word(b + 4), (int)word(b));
    }
    __device__ __forceinline__ int u16(size_t b) const
    {
        const uint32_t x = word(b);
        return (b & 2) ? (int)(x >> 16) : (int)(x & 0xFFFFu);
    }
    __device__ __forceinline__ int u8(size_t b) const
    {
        return (int)((word(b) >> (8 * (b & 3))) & 0xFFu);
    }
};
#define RXO(field) offsetof(RxnF32, field)

template <bool ANN>
__global__ void __launch_bounds__(32 * kF32Warps)
k_source_f32(MechViewF32 mv, IntView iv, KcAnnView av, int64_t n, int cpw,
             const float *__restrict__ T, const float *__restrict__ P,
             const float *__restrict__ Y, int64_t ldY, float *__restrict__ om, int64_t ldO)
{
    extern __shared__ float smem32[];
    const int ns = mv.ns, nr = mv.nr, lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
    const int per_warp = 32 * kCellScalars + 5 * ns + nr + (ANN ? 2 * kAnnMaxHidden : 0);
    float *cs = smem32 + (size_t)wb * per_warp;    // [32 cells][kCellScalars]
    float *sE = cs + 32 * kCellScalars;            // integer part of log2 z_k (exact)
    float *sF = sE + ns;                           // log2 of the mantissa of z_k, in [-1, 0)
    float *sX = sF + ns;                           // X_k (third-body sums)
    float *sGh = sX + ns;                          // -g_k/(RT) in log2 units, double-float
    float *sGl = sGh + ns;
    float *sQ = sGl + ns;                          // q_net per reaction
    float *sH = sQ + nr;                           // ANN: two layers of hidden units
    const int64_t i0 = ((int64_t)blockIdx.x * kF32Warps + wb) * cpw;
    if (i0 >= n) return;

    // ---- per-cell features of the warp's cells, one lane per cell (FP64 -> double-float)
    {
        const int64_t i = i0 + lane;
        float *c = cs + lane * kCellScalars;
        if (lane < cpw && i < n) {
            const float Tf = T[i], Pf = P[i];
            const double Td = (double)Tf, lg2Td = log2(Td), taud = Td * 1e-3;
            const df lg2T = df_from_double(lg2Td), invT = df_from_double(1.0 / Td);
            const df p2 = df_from_double(taud), p3 = df_from_double(taud * taud);
            const df p4 = df_from_double(taud * taud * taud);
            const df p5 = df_from_double(taud * taud * taud * taud);
            const df lgct = df_from_double(log2((double)Pf) - log2(kR) - lg2Td);  // log2 c_tot
            const float v[kCellScalars] = {lg2T.h, lg2T.l, invT.h, invT.l, p2.h, p2.l, p3.h, p3.l,
                                           p4.h,   p4.l,   p5.h,   p5.l,   lgct.h, lgct.l, Tf,
                                           Tf >= mv.t_mid ? 1.0f : 0.0f};
#pragma unroll
            for (int q = 0; q < kCellScalars; ++q) c[q] = v[q];
        }
    }
    __syncwarp();

    for (int cc = 0; cc < cpw && i0 + cc < n; ++cc) {
        const int64_t i = i0 + cc;
        const float *c = cs + cc * kCellScalars;
        const df lg2T = mkdf(c[0], c[1]), invT = mkdf(c[2], c[3]);
        const df lgct = mkdf(c[12], c[13]);
        const float Tf = c[14];
        const int rg = c[15] != 0.0f ? 1 : 0;
        // ---- species: z_k, log2 z_k, Gibbs layer (Eq. 10), sum_k z_k
        df zsum = mkdf(0.0f, 0.0f);
        for (int k = lane; k < ns; k += 32) {
            float y = Y[i * ldY + k];
            const float z = (y > 0.0f ? y : 0.0f) * mv.spec[k].invW;
            zsum = df_add_f(zsum, z);
            sX[k] = z;
            if (z > 0.0f) {
                int ex;
                const float m = frexpf(z, &ex);     // z = m 2^ex, m in [0.5, 1)
                sE[k] = (float)ex;
                sF[k] = log2f(m);
            } else {
                sE[k] = kLg2Floor;
                sF[k] = 0.0f;
            }
            if (!ANN) {
                const df phi[7] = {mkdf(1.0f, 0.0f), lg2T,           mkdf(c[4], c[5]),
                                   mkdf(c[6], c[7]),  mkdf(c[8], c[9]), mkdf(c[10], c[11]), invT};
                const float2 *g = mv.spec[k].gl[rg];
                df G = mkdf(g[0]);
                for (int m = 1; m < 7; ++m) G = df_add(G, df_mul(mkdf(g[m]), phi[m]));
                sGh[k] = G.h;
                sGl[k] = G.l;
            }
        }
        zsum = df_warp_sum(zsum);
        const bool any = zsum.h > 0.0f;
        const float inv_sum = any ? 1.0f / zsum.h : 0.0f;
        for (int k = lane; k < ns; k += 32) sX[k] *= inv_sum;    // X_k = z_k / sum_k z_k
        // log2 X_k = log2 z_k - log2 sum_k z_k: the second term enters every reaction through
        // its order, together with log2 c_tot
        const df ls = any ? df_log2(zsum) : mkdf(0.0f, 0.0f);
        const df lgcn = df_add(lgct, mkdf(-ls.h, -ls.l));
        const df lgpRT = df_add(mkdf(mv.lg2_pref_R), mkdf(-lg2T.h, -lg2T.l));   // log2(p_ref/RT)
        int cur = 0;
        if (ANN) {
            const float x = (logf(Tf) - av.x_mean) * av.x_inv_std;
            if (lane < av.nh) sH[lane] = ann_act(fmaf(av.w_in[lane], x, av.b_in[lane]), av.act);
            for (int l = 0; l + 1 < av.nl; ++l) {
                __syncwarp();
                const float *W = av.w_hid + (size_t)l * av.nh * av.nh;
                if (lane < av.nh) {
                    float a = av.b_hid[l * av.nh + lane];
                    for (int h = 0; h < av.nh; ++h)
                        a = fmaf(W[h * av.nh + lane], sH[cur * kAnnMaxHidden + h], a);
                    sH[(cur ^ 1) * kAnnMaxHidden + lane] = ann_act(a, av.act);
                }
                cur ^= 1;
            }
        }
        __syncwarp();
        // ---- reactions, one slot per lane
        for (int sl = lane; sl < iv.n_slots; sl += 32) {
            const int j = iv.order[sl];
            if (j < 0) continue;
            const RxnW R{mv.rxn_t + sl, mv.n_slots};
            // Arrhenius layer, log2 k_inf (Eq. 6)
            const df tf = df_add(df_add(R.d2(RXO(kf)), df_mul(R.d2(RXO(kf) + 8), lg2T)),
                                 df_mul(R.d2(RXO(kf) + 16), invT));
            // third-body / falloff factor, log2 (Sec. 2.4)
            df fac = mkdf(0.0f, 0.0f);
            bool dead = false;
            const int kind = R.i(RXO(kind));
            if (kind != 0) {
                float s = 1.0f;                    // M / c_tot = 1 + sum_k (eff_k - 1) X_k
                const int tb1 = R.i(RXO(tb_end));
                for (int t = R.i(RXO(tb_begin)); t < tb1; ++t) s = fmaf(mv.tb_e[t], sX[mv.tb_sp[t]], s);
                if (!(s > 0.0f)) {
                    dead = true;
                } else {
                    const df lgM = df_add_f(lgct, log2f(s));
                    if (kind == 1) {
                        fac = lgM;
                    } else {
                        df t0 = df_add(df_add(R.d2(RXO(k0)), df_mul(R.d2(RXO(k0) + 8), lg2T)),
                                       df_mul(R.d2(RXO(k0) + 16), invT));
                        df lPr = df_add(df_add(t0, mkdf(-tf.h, -tf.l)), lgM);   // log2 Pr
                        // log2(Pr / (1 + Pr)) without cancellation on either side of Pr = 1
                        if (lPr.h < 0.0f)
                            fac = df_add_f(lPr, -log2f(1.0f + exp2f(lPr.h)));
                        else
                            fac = mkdf(-log2f(1.0f + exp2f(-lPr.h)), 0.0f);
                        if (kind == 3) {
                            const float tr4 = R.f(RXO(troe) + 16);
                            float Fc = R.f(RXO(troe)) * expf(-Tf * R.f(RXO(troe) + 8)) +
                                       R.f(RXO(troe) + 4) * expf(-Tf * R.f(RXO(troe) + 12));
                            if (tr4 > 0.0f) Fc += expf(-tr4 / Tf);
                            const float lFc = log10f(Fc);
                            const float c1 = -0.4f - 0.67f * lFc, nn = 0.75f - 1.27f * lFc;
                            const float x = (lPr.h + lPr.l) * 0.30102999566398120f + c1;
                            const float f1 = x / (nn - 0.14f * x);
                            fac = df_add_f(fac, lFc / (1.0f + f1 * f1) * 3.3219280948873623f);
                        }
                    }
                }
            }
            float qn = 0.0f;
            if (!dead) {
                // forward: tf + ord' log2(c_tot / sum z) + sum nu' log2 z + factor
                float ei = 0.0f, fs = 0.0f;
                const int nf = R.i(RXO(nf)), nrr = R.i(RXO(nr));
                for (int t = 0; t < nf; ++t) {
                    const int k = R.u16(RXO(spf) + 2 * t);
                    const float nu = (float)R.u8(RXO(nuf) + t);
                    ei = fmaf(nu, sE[k], ei);
                    fs = fmaf(nu, sF[k], fs);
                }
                df xf = df_add(df_add(tf, df_mul_f(lgcn, (float)R.i(RXO(ordf)))), fac);
                xf = df_add_f(df_add_f(xf, ei), fs);
                qn = df_exp2(xf);
                if (R.i(RXO(rev))) {
                    df lkc;
                    float er = 0.0f, fr = 0.0f;
                    if (ANN) {
                        // ln K_c = y_mean + y_std (b + sum_h w_h a_h) (Eq. 14), in log2 units
                        float a = av.b_out[j];
                        for (int h = 0; h < av.nh; ++h)
                            a = fmaf(av.w_out[(size_t)h * nr + j], sH[cur * kAnnMaxHidden + h], a);
                        lkc = mkdf(fmaf(av.y_std[j], a, av.y_mean[j]) * 1.4426950408889634f, 0.0f);
                        for (int t = 0; t < nrr; ++t) {
                            const int k = R.u16(RXO(spr) + 2 * t);
                            const float nu = (float)R.u8(RXO(nur) + t);
                            er = fmaf(nu, sE[k], er);
                            fr = fmaf(nu, sF[k], fr);
                        }
                    } else {
                        // log2 K_c = sum_k nu_kj (-g_k/RT) + dnu log2(p_ref/RT) (Eqs. 8-9)
                        lkc = df_mul_f(lgpRT, (float)R.i(RXO(dnu)));
                        for (int t = 0; t < nrr; ++t) {
                            const int k = R.u16(RXO(spr) + 2 * t);
                            const float nu = (float)R.u8(RXO(nur) + t);
                            lkc = df_add(lkc, df_mul_f(mkdf(sGh[k], sGl[k]), nu));
                            er = fmaf(nu, sE[k], er);
                            fr = fmaf(nu, sF[k], fr);
                        }
                        for (int t = 0; t < nf; ++t) {
                            const int k = R.u16(RXO(spf) + 2 * t);
                            lkc = df_add(lkc, df_mul_f(mkdf(sGh[k], sGl[k]),
                                                       -(float)R.u8(RXO(nuf) + t)));
                        }
                    }
                    df xr = df_add(df_add(tf, df_mul_f(lgcn, (float)R.i(RXO(ordr)))), fac);
                    xr = df_add(xr, mkdf(-lkc.h, -lkc.l));
                    xr = df_add_f(df_add_f(xr, er), fr);
                    qn -= df_exp2(xr);
                }
            }
            sQ[j] = qn;
        }
        __syncwarp();
        // ---- omega_k = sum_j (nu''_kj - nu'_kj) q_net,j (Eq. 2), compensated, reaction order;
        // the species are spread over the lanes by entry count
        for (int a = mv.lane_ptr[lane]; a < mv.lane_ptr[lane + 1]; ++a) {
            const int k = mv.lane_sp[a];
            float ws = 0.0f, wc = 0.0f;
            for (int e = mv.col_ptr[k]; e < mv.col_ptr[k + 1]; ++e) {
                const df t = two_sum(ws, mv.col_nu[e] * sQ[mv.col_rxn[e]]);
                ws = t.h;
                wc += t.l;
            }
            om[i * ldO + k] = ws + wc;
        }
    }
}

// ---------------------------------------------------------------------------------------
// FP64
// ---------------------------------------------------------------------------------------

// One warp per cell, cpw cells per warp, as k_source_f32, in plain FP64 and natural-log
// units: the lane-per-cell pass computes ln T, 1/T, tau, c_tot; per cell the lanes take the
// species (C_k = c_tot z_k / sum z, ln C_k; -inf for an absent species), the reactions
// (Arrhenius layer, third-body / falloff factor, the FP64 folded Gibbs polynomial of the
// reaction's T range, exp of both sides) and omega by the species-major gather.
constexpr int kF64Warps = 8;                   // warps per block
constexpr int kCell64 = 6;                     // per-cell scalars kept in shared memory
#define RXO64(field) offsetof(RxnF64, field)

__global__ void __launch_bounds__(32 * kF64Warps)
k_source_f64(MechViewF64 mv, IntView iv, int64_t n, int cpw, const double *__restrict__ T,
             const double *__restrict__ P, const double *__restrict__ Y, int64_t ldY,
             double *__restrict__ om, int64_t ldO)
{
    extern __shared__ double smem64[];
    const int ns = mv.ns, nr = mv.nr, lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
    const int per_warp = 32 * kCell64 + 2 * ns + nr;
    double *cs = smem64 + (size_t)wb * per_warp;   // [cells][kCell64]
    double *sC = cs + 32 * kCell64;                // C_k
    double *sL = sC + ns;                          // ln C_k
    double *sQ = sL + ns;                          // q_net per reaction
    const int64_t i0 = ((int64_t)blockIdx.x * kF64Warps + wb) * cpw;
    if (i0 >= n) return;
    {
        const int64_t i = i0 + lane;
        if (lane < cpw && i < n) {
            const double Ti = T[i], Pi = P[i];
            double *c = cs + lane * kCell64;
            c[0] = log(Ti);
            c[1] = 1.0 / Ti;
            c[2] = Ti * 1e-3;
            c[3] = Pi / (kR * Ti);                 // c_tot
            c[4] = Ti;
            c[5] = Ti >= mv.t_mid ? 1.0 : 0.0;
        }
    }
    __syncwarp();
    for (int cc = 0; cc < cpw && i0 + cc < n; ++cc) {
        const int64_t i = i0 + cc;
        const double *c = cs + cc * kCell64;
        const double lnT = c[0], invT = c[1], tau = c[2], ctot = c[3], Ti = c[4];
        const int rg = c[5] != 0.0 ? 1 : 0;
        // ---- species: C_k = c_tot z_k / sum_k z_k, ln C_k
        double zs = 0.0;
        for (int k = lane; k < ns; k += 32) {
            const double y = Y[i * ldY + k];
            const double z = (y > 0.0 ? y : 0.0) * mv.invW[k];
            sC[k] = z;
            zs += z;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) zs += __shfl_xor_sync(0xffffffffu, zs, off);
        const double scale = zs > 0.0 ? ctot / zs : 0.0;
        for (int k = lane; k < ns; k += 32) {
            const double cv = sC[k] * scale;
            sC[k] = cv;
            sL[k] = log(cv);                       // -inf for an absent species
        }
        __syncwarp();
        // ---- reactions, one slot per lane
        for (int sl = lane; sl < mv.n_slots; sl += 32) {
            const int j = iv.order[sl];
            if (j < 0) continue;
            const RxnW R{mv.rxn_t + sl, mv.n_slots};
            const double lkinf = R.dbl(RXO64(lnA)) + R.dbl(RXO64(b)) * lnT -
                                 R.dbl(RXO64(EoR)) * invT;          // Eq. 6
            double lfac = 0.0;                     // Sec. 2.4
            const int kind = R.i(RXO64(kind));
            if (kind != 0) {
                double M = ctot;                   // sum_k eff_k C_k = c_tot + sum_k (eff_k - 1) C_k
                const int tb1 = R.i(RXO64(tb_end));
                for (int t = R.i(RXO64(tb_begin)); t < tb1; ++t) M += mv.tb_e[t] * sC[mv.tb_sp[t]];
                if (kind == 1) {
                    lfac = log(M);
                } else {
                    const double lk0 = R.dbl(RXO64(low)) + R.dbl(RXO64(low) + 8) * lnT -
                                       R.dbl(RXO64(low) + 16) * invT;
                    const double Pr = exp(lk0 - lkinf) * M;
                    if (Pr > 0.0) {
                        lfac = log(Pr / (1.0 + Pr));
                        if (kind == 3) {
                            const size_t ot = RXO64(troe);
                            const double t4 = R.dbl(ot + 32);
                            double Fc = R.dbl(ot) * exp(-Ti * R.dbl(ot + 16)) +
                                        R.dbl(ot + 8) * exp(-Ti * R.dbl(ot + 24));
                            if (t4 > 0.0) Fc += exp(-t4 * invT);
                            const double lFc = log10(Fc);
                            const double c1 = -0.4 - 0.67 * lFc, nn = 0.75 - 1.27 * lFc;
                            const double x = log10(Pr) + c1;
                            const double f1 = x / (nn - 0.14 * x);
                            lfac += lFc / (1.0 + f1 * f1) * 2.302585092994045684;
                        }
                    } else {
                        lfac = -INFINITY;
                    }
                }
            }
            const size_t ok = RXO64(kc) + (size_t)rg * 56;     // Eqs. 9-11, folded
            const double lKc = R.dbl(ok) + R.dbl(ok + 8) * lnT +
                               tau * (R.dbl(ok + 16) +
                                      tau * (R.dbl(ok + 24) + tau * (R.dbl(ok + 32) + tau * R.dbl(ok + 40)))) +
                               R.dbl(ok + 48) * invT;
            double sf = lkinf + lfac, sr = lkinf + lfac - lKc;
            const int nf = R.i(RXO64(nf)), nrr = R.i(RXO64(nr));
            for (int t = 0; t < nf; ++t) sf += R.u8(RXO64(nuf) + t) * sL[R.u16(RXO64(spf) + 2 * t)];
            for (int t = 0; t < nrr; ++t) sr += R.u8(RXO64(nur) + t) * sL[R.u16(RXO64(spr) + 2 * t)];
            const double qf = exp(sf);
            const double qr = R.i(RXO64(rev)) ? exp(sr) : 0.0;
            sQ[j] = qf - qr;
        }
        __syncwarp();
        // ---- omega_k = sum_j (nu''_kj - nu'_kj) q_net,j (Eq. 2), reaction order
        for (int a = mv.lane_ptr[lane]; a < mv.lane_ptr[lane + 1]; ++a) {
            const int k = mv.lane_sp[a];
            double w = 0.0;
            for (int e = mv.col_ptr[k]; e < mv.col_ptr[k + 1]; ++e)
                w += (double)mv.col_nu[e] * sQ[mv.col_rxn[e]];
            om[i * ldO + k] = w;
        }
    }
}

// ---------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------

constexpr size_t kMaxDynSmem = 227 * 1024;

// Resident warps of a kernel on the current device (SMs x blocks per SM x warps per block),
// queried once per mechanism and path.
template <typename K>
static int64_t resident_warps(const chem_mech *m, int slot, K kern, int warps_per_block, size_t smem)
{
    int w = const_cast<chem_mech *>(m)->simt_warps[slot].load(std::memory_order_relaxed);
    if (w <= 0) {
        int dev = 0, nsm = 0, blocks = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, 32 * warps_per_block, smem);
        w = (nsm > 0 ? nsm : 1) * (blocks > 0 ? blocks : 1) * warps_per_block;
        const_cast<chem_mech *>(m)->simt_warps[slot].store(w, std::memory_order_relaxed);
    }
    return w;
}

// Cells per warp: 32 when the batch fills every resident warp 32 times over, else just
// enough to cover the batch with the resident warps.
static int cells_per_warp(int64_t n, int64_t warps)
{
    const int64_t cpw = (n + warps - 1) / warps;
    return (int)(cpw < 1 ? 1 : cpw > 32 ? 32 : cpw);
}

chem_status launch_source_fp64(const chem_mech *m, int64_t n, const double *T, const double *P,
                               const double *Y, int64_t ldY, double *om, int64_t ldO,
                               cudaStream_t s)
{
    static SmemOptIn opt;
    if (n <= 0) return CHEM_OK;
    const size_t smem =
        sizeof(double) * kF64Warps * (32 * (size_t)kCell64 + 2 * (size_t)m->ns + (size_t)m->nr);
    if (smem > kMaxDynSmem)
        return set_error(CHEM_EUNSUPPORTED, "fp64: %d species / %d reactions exceed the SIMT kernel",
                         m->ns, m->nr);
    chem_status st = opt.ensure((const void *)k_source_f64, (int)kMaxDynSmem, false, "fp64");
    if (st != CHEM_OK) return st;
    const int cpw = cells_per_warp(n, resident_warps(m, 0, k_source_f64, kF64Warps, smem));
    const int64_t per_block = (int64_t)cpw * kF64Warps;
    st = launch_opted(opt, (const void *)k_source_f64, (int)kMaxDynSmem, "fp64", [&] {
        k_source_f64<<<(unsigned)((n + per_block - 1) / per_block), 32 * kF64Warps, smem, s>>>(
            m->v64, m->vint, n, cpw, T, P, Y, ldY, om, ldO);
    });
    if (st == CHEM_OK) g_launches.fetch_add(1);
    return st;
}

static size_t f32_warp_floats(const chem_mech *m, bool ann)
{
    return 32 * (size_t)kCellScalars + 5 * (size_t)m->ns + (size_t)m->nr +
           (ann ? 2 * (size_t)kAnnMaxHidden : 0);
}

template <bool ANN>
static chem_status launch_f32(const chem_mech *m, const KcAnnView &av, int64_t n, const float *T,
                              const float *P, const float *Y, int64_t ldY, float *om,
                              int64_t ldO, cudaStream_t s, const char *name)
{
    static SmemOptIn opt;
    if (n <= 0) return CHEM_OK;
    const size_t smem = sizeof(float) * kF32Warps * f32_warp_floats(m, ANN);
    if (smem > kMaxDynSmem)
        return set_error(CHEM_EUNSUPPORTED, "%s: %d species / %d reactions exceed the SIMT kernel",
                         name, m->ns, m->nr);
    chem_status st = opt.ensure((const void *)k_source_f32<ANN>, (int)kMaxDynSmem, false, name);
    if (st != CHEM_OK) return st;
    const int cpw =
        cells_per_warp(n, resident_warps(m, ANN ? 2 : 1, k_source_f32<ANN>, kF32Warps, smem));
    const int64_t per_block = (int64_t)cpw * kF32Warps;
    st = launch_opted(opt, (const void *)k_source_f32<ANN>, (int)kMaxDynSmem, name, [&] {
        k_source_f32<ANN><<<(unsigned)((n + per_block - 1) / per_block), 32 * kF32Warps, smem, s>>>(
            m->v32, m->vint, av, n, cpw, T, P, Y, ldY, om, ldO);
    });
    if (st == CHEM_OK) g_launches.fetch_add(1);
    return st;
}

chem_status launch_source_fp32(const chem_mech *m, int64_t n, const float *T, const float *P,
                               const float *Y, int64_t ldY, float *om, int64_t ldO,
                               cudaStream_t s)
{
    if (m->vt.ok) return launch_source_fp32_t(m, n, T, P, Y, ldY, om, ldO, s);
    KcAnnView none;
    memset(&none, 0, sizeof none);
    return launch_f32<false>(m, none, n, T, P, Y, ldY, om, ldO, s, "fp32");
}

chem_status launch_source_fp32_warp(const chem_mech *m, int64_t n, const float *T, const float *P,
                                    const float *Y, int64_t ldY, float *om, int64_t ldO,
                                    cudaStream_t s)
{
    KcAnnView none;
    memset(&none, 0, sizeof none);
    return launch_f32<false>(m, none, n, T, P, Y, ldY, om, ldO, s, "fp32 warp per cell");
}

chem_status launch_source_fp32_ann(const chem_mech *m, const KcAnnView &av, int64_t n,
                                   const float *T, const float *P, const float *Y, int64_t ldY,
                                   float *om, int64_t ldO, cudaStream_t s)
{
    return launch_f32<true>(m, av, n, T, P, Y, ldY, om, ldO, s, "fp32 ann");
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
