// kern_f32t.cu -- FP32 source term, one thread per cell (Eqs. 2-11, Sec. 2.4).
//
// A warp takes 32 cells, one per lane, and walks the mechanism's reactions with all lanes on
// the same reaction: every table read is a broadcast and every branch on the reaction's kind
// is warp-uniform.  Per cell and species, shared memory holds
//   P_k = log2 C_k                                  (Eq. 3 in log2 units)
//   F_k = -g_k/(R T) log2 e + log2(p_ref / (R T))   (the Gibbs layer, Eqs. 8-11)
// so that for reaction j, with log2 K_c = sum_k nu_kj F_k,
//   x_f = log2 k_f + fac + sum_k nu'_kj P_k
//   x_r = log2 k_f + fac + sum_k nu''_kj (P_k - F_k) + sum_k nu'_kj F_k
//   q_net = 2^x_f - 2^x_r,   omega_k += (nu''_kj - nu'_kj) q_net      (Eqs. 2-4, 7)
// where fac is log2 of the third-body concentration or of the falloff factor (Sec. 2.4).
//
// Precision: every exponent is a pair (H, L), H a multiple of 2^-12 and L small.  Heads of
// the per-species terms and of the products of a reaction's temperature coefficients with
// the cell's centred temperature features are put on that grid, so the sums of heads with
// small integer stoichiometric coefficients are exact in FP32; only L carries rounding, at
// the magnitude of L, and 2^(H + L) is taken as 2^H 2^L.  The per-cell temperature features
// are double-float (log2 by an atanh series, 1/T with its Newton residual); the bounded
// third-body and falloff factors use the MUFU exp2 / log2; the Gibbs polynomial is expanded
// about its T range's own centre.  omega accumulates in FP32 in the processing order
// (per-cell error ~8e-7 of max |omega| at 53/325).
//
// Layout: one block of W warps per SM-sized share of the batch.  The block stages the species
// table, the third-body lists and the falloff parameters once, and the reaction records in
// double-buffered chunks of 16 (loaded one chunk ahead); each warp owns its P/F rows (12
// bytes per species and cell: the heads in FP32, the remainders, below 2^-12, in FP16) and
// its omega tile.  Reactions are grouped by kind and shape (at most two or three species per
// side) into quads whose net species are distinct where possible (chem_quads.h) and taken
// four at a time, elementary ones eight at a time (two quads), with fixed-shape code, so
// that their exponent chains overlap and each quad updates omega in one round trip.
#include <math.h>
#include <stddef.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <vector>

#include <cuda_fp16.h>

#include "chem_f32t_tables.h"

namespace chem {

using namespace f32t;

// Tables of the kernel from the descriptor; a mechanism outside the kernel's limits keeps
// m->vt.ok false and the FP32 source term then runs the warp-per-cell kernel.
chem_status f32t_build_tables(chem_mech *m, const chem_mech_desc *d)
{
    m->vt = F32TView{};
    m->d_f32t = nullptr;
    Tables t;
    if (!build_tables(d, t)) return CHEM_OK;
    const int ns = d->n_species;
    const std::vector<RxnT> &rx = t.rx;
    const std::vector<SpecT> &sp = t.sp;
    const std::vector<int2> &tb = t.tb;
    const std::vector<FallT> &fall = t.fall;
    auto align = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t ntb = tb.empty() ? 1 : tb.size(), nfa = fall.empty() ? 1 : fall.size();
    const size_t o_rx = 0, o_sp = align(sizeof(RxnT) * rx.size()),
                 o_tb = align(o_sp + sizeof(SpecT) * ns), o_fa = align(o_tb + sizeof(int2) * ntb),
                 total = align(o_fa + sizeof(FallT) * nfa);
    std::vector<unsigned char> h(total, 0);
    memcpy(h.data() + o_rx, rx.data(), sizeof(RxnT) * rx.size());
    memcpy(h.data() + o_sp, sp.data(), sizeof(SpecT) * ns);
    if (!tb.empty()) memcpy(h.data() + o_tb, tb.data(), sizeof(int2) * tb.size());
    if (!fall.empty()) memcpy(h.data() + o_fa, fall.data(), sizeof(FallT) * fall.size());
    F32TView v = t.v;
    void *dp = nullptr;
    cudaError_t e = cudaMalloc(&dp, total);
    if (e != cudaSuccess) return set_error(CHEM_ENOMEM, "cudaMalloc(%zu): %s", total, cudaGetErrorString(e));
    e = cudaMemcpy(dp, h.data(), total, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(dp);
        return set_error(CHEM_ECUDA, "cudaMemcpy: %s", cudaGetErrorString(e));
    }
    unsigned char *base = (unsigned char *)dp;
    v.rxn = (const RxnT *)(base + o_rx);
    v.spec = (const SpecT *)(base + o_sp);
    v.tb = (const int2 *)(base + o_tb);
    v.fall = (const FallT *)(base + o_fa);
    v.ok = true;
    m->vt = v;
    m->d_f32t = dp;
    m->device_bytes += total;
    return CHEM_OK;
}

void f32t_free_tables(chem_mech *m)
{
    if (m->d_f32t) cudaFree(m->d_f32t);
    m->d_f32t = nullptr;
    m->vt.ok = false;
}

namespace {

__device__ __forceinline__ float grid12(float x) { return __fsub_rn(__fadd_rn(x, kGridAdd), kGridAdd); }

// (P_h, P_l, F_h, F_l) of the species row at byte offset off; pfh / pfl: this lane's
// float2 / half2 columns of row 0
__device__ __forceinline__ float4 load_pf(const char *pfh, const char *pfl, int off)
{
    const float2 h = *(const float2 *)(pfh + off);
    const float2 l = __half22float2(*(const __half2 *)(pfl + off));
    return make_float4(h.x, l.x, h.y, l.y);
}

// 2^x, flushed to zero below the normal range (MUFU exp2)
__device__ __forceinline__ float ex2_ftz(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// log2 x (MUFU log2) for the bounded factors of the third-body and falloff terms
__device__ __forceinline__ float lg2_approx(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// (H, L) += c d for a double-float coefficient c and a double-float cell feature d: the
// rounded product goes to the 2^-12 grid in H, its remainder and rounding error to L.
__device__ __forceinline__ void acc_prod(float &H, float &L, float ch, float cl, float dh, float dl)
{
    const float p = __fmul_rn(ch, dh);
    const float e = fmaf(ch, dl, fmaf(cl, dh, fmaf(ch, dh, -p)));
    const float ph = grid12(p);
    H = __fadd_rn(H, ph);
    L = __fadd_rn(L, __fadd_rn(__fsub_rn(p, ph), e));
}

// double-float arithmetic (Knuth two-sum, Dekker fast two-sum, FMA two-product); the
// explicit _rn forms keep the compiler from contracting them
struct dflt {
    float h, l;
};
__device__ __forceinline__ dflt two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ dflt fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dflt df_add(dflt a, dflt b)
{
    const dflt s = two_sum(a.h, b.h);
    return fast_two_sum(s.h, __fadd_rn(__fadd_rn(a.l, b.l), s.l));
}
__device__ __forceinline__ dflt df_mul(dflt a, dflt b)
{
    const float p = __fmul_rn(a.h, b.h);
    return fast_two_sum(p, fmaf(a.h, b.l, fmaf(a.l, b.h, fmaf(a.h, b.h, -p))));
}
__device__ __forceinline__ dflt df_neg(dflt a) { return {-a.h, -a.l}; }
__device__ __forceinline__ dflt df_of(float2 v) { return {v.x, v.y}; }

// log2 of a positive normal float as a double-float: x = 2^e m with m in [0.75, 1.5),
// ln m = 2 atanh(s) = 2 (s + s^3/3 + s^5/5 + ...), s = (m - 1) / (m + 1), |s| <= 1/5; the
// series to s^13 leaves < 1e-11, s carries its division residual
__device__ __forceinline__ dflt df_log2f(float x, dflt log2e)
{
    const int bits = __float_as_int(x);
    int e = ((bits >> 23) & 0xFF) - 127;
    float m = __int_as_float((bits & 0x007FFFFF) | 0x3F800000);      // [1, 2)
    if (m >= 1.5f) {
        m *= 0.5f;
        e += 1;
    }
    const float num = __fsub_rn(m, 1.0f);                               // exact
    const dflt den = two_sum(m, 1.0f);
    const float sh = __fdiv_rn(num, den.h);
    const float sl = __fdiv_rn(__fsub_rn(fmaf(-sh, den.h, num), __fmul_rn(sh, den.l)), den.h);
    const float s2 = __fmul_rn(sh, sh);
    float t = fmaf(s2, 1.0f / 13.0f, 1.0f / 11.0f);
    t = fmaf(s2, t, 1.0f / 9.0f);
    t = fmaf(s2, t, 1.0f / 7.0f);
    t = fmaf(s2, t, 1.0f / 5.0f);
    t = fmaf(s2, t, 1.0f / 3.0f);
    t = __fmul_rn(t, s2);                                               // s^2/3 + s^4/5 + ...
    const dflt lnm = fast_two_sum(2.0f * sh, fmaf(2.0f * sh, t, 2.0f * sl));
    return df_add({(float)e, 0.0f}, df_mul(lnm, log2e));
}

// Split a double-float onto the grid: head exact in float, remainder rounded.
__device__ __forceinline__ void grid_split(dflt x, float &h, float &r)
{
    h = grid12(x.h);
    r = __fadd_rn(__fsub_rn(x.h, h), x.l);
}

struct CellF {
    float d1h, d2h, d2l;                     // centred log2 T and 1/T
    float ctH, ctR;                          // log2 c_tot on the grid
    float Tf, invT;
};

// omega_k += (nu''_kj - nu'_kj) q_net,j (Eq. 2); om: this lane's column of the omega tile.
// A reaction's net species are distinct (unused entries add 0 to the zero row), so all its
// values are read before any is written: one shared-memory round trip per reaction.
template <int NN>
__device__ __forceinline__ void scatter(const RxnT &R, char *om, float q)
{
    const int4 *E = (const int4 *)R.ent;
    int off[NN];
    float nu[NN], v[NN];
#pragma unroll
    for (int t = 0; t < NN; ++t) {
        const int4 w = E[rxnt_net(t) / 2];
        off[t] = rxnt_net(t) % 2 ? w.z : w.x;
        nu[t] = __int_as_float(rxnt_net(t) % 2 ? w.w : w.y);
        v[t] = *(const float *)(om + off[t]);
    }
#pragma unroll
    for (int t = 0; t < NN; ++t) *(float *)(om + off[t]) = fmaf(nu[t], q, v[t]);
}

// entry (offset, coefficient) of pair index `pair` of record R
__device__ __forceinline__ void entry(const RxnT &R, int pair, int &off, float &nu)
{
    const int4 w = ((const int4 *)R.ent)[pair / 2];
    off = pair % 2 ? w.z : w.x;
    nu = __int_as_float(pair % 2 ? w.w : w.y);
}

// omega update of a quad: one round when the quad's net species are pairwise distinct (meta
// bit 3), else one round per reaction
template <int NN>
__device__ __forceinline__ void scatter_quad(const RxnT *R, char *om, const float *q)
{
    if (R[0].meta & 8u) {
        int off[kQuad][NN];
        float nu[kQuad][NN], v[kQuad][NN];
#pragma unroll
        for (int u = 0; u < kQuad; ++u)
#pragma unroll
            for (int t = 0; t < NN; ++t) {
                entry(R[u], rxnt_net(t), off[u][t], nu[u][t]);
                v[u][t] = *(const float *)(om + off[u][t]);
            }
#pragma unroll
        for (int u = 0; u < kQuad; ++u)
#pragma unroll
            for (int t = 0; t < NN; ++t) *(float *)(om + off[u][t]) = fmaf(nu[u][t], q[u], v[u][t]);
    } else {
#pragma unroll
        for (int u = 0; u < kQuad; ++u) scatter<NN>(R[u], om, q[u]);
    }
}

// kQuad reactions of one group (KIND 0 elementary, 1 third-body, 2 Lindemann, 3 Troe),
// written step by step across the four so that consecutive instructions are independent
template <int NF, int NR, int NN, int KIND, int U = kQuad>
__device__ __forceinline__ void quad(const RxnT *R, const char *pfh, const char *pfl, char *om,
                                     const int2 *tb, const FallT *fall, const CellF &c)
{
    static_assert(U % kQuad == 0 && (KIND == 0 || U == kQuad), "quads of elementary reactions pair up");
    float4 kf[U];
    float b[U], rb[U], p[U], e[U], ph[U], xfH[U], xfL[U], xrH[U], xrL[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        kf[u] = R[u].kf;
        const float4 hd = *(const float4 *)&R[u].b;
        b[u] = hd.x;
        rb[u] = hd.w;
    }
    // log2 k_inf (Eq. 6): head of (-E/R log2 e) d2 on the grid, the rest in L
#pragma unroll
    for (int u = 0; u < U; ++u) p[u] = __fmul_rn(kf[u].z, c.d2h);
#pragma unroll
    for (int u = 0; u < U; ++u) e[u] = fmaf(kf[u].z, c.d2h, -p[u]);
#pragma unroll
    for (int u = 0; u < U; ++u) e[u] = fmaf(kf[u].w, c.d2h, e[u]);
#pragma unroll
    for (int u = 0; u < U; ++u) e[u] = fmaf(kf[u].z, c.d2l, e[u]);
#pragma unroll
    for (int u = 0; u < U; ++u) ph[u] = __fadd_rn(p[u], kGridAdd);
#pragma unroll
    for (int u = 0; u < U; ++u) ph[u] = __fsub_rn(ph[u], kGridAdd);
#pragma unroll
    for (int u = 0; u < U; ++u) xfL[u] = fmaf(b[u], c.d1h, kf[u].y);
#pragma unroll
    for (int u = 0; u < U; ++u) xfH[u] = __fadd_rn(kf[u].x, ph[u]);
#pragma unroll
    for (int u = 0; u < U; ++u) e[u] = __fadd_rn(__fsub_rn(p[u], ph[u]), e[u]);
#pragma unroll
    for (int u = 0; u < U; ++u) xfL[u] = __fadd_rn(xfL[u], e[u]);
    bool live[U];
#pragma unroll
    for (int u = 0; u < U; ++u) live[u] = true;
    if (KIND != 0) {
        // M / c_tot = 1 + sum_k (eff_k - 1) X_k, X_k = 2^(P_k - log2 c_tot)      (Sec. 2.4);
        // the quad's lists interleaved [entry][reaction], padded with zero entries
        float s[U];
#pragma unroll
        for (int u = 0; u < U; ++u) s[u] = 1.0f;
        const uint32_t tw = R[0].tb;
        const int2 *te = tb + (tw & 0xFFFFu);
        const int nit = (int)(tw >> 16);
        for (int it = 0; it < nit; ++it) {
            int2 en[U];
            float2 pp[U];
#pragma unroll
            for (int u = 0; u < U; ++u) en[u] = te[it * U + u];
#pragma unroll
            for (int u = 0; u < U; ++u)
                pp[u] = make_float2(((const float2 *)(pfh + en[u].x))->x,
                                    __low2float(*(const __half2 *)(pfl + en[u].x)));
#pragma unroll
            for (int u = 0; u < U; ++u)
                s[u] = fmaf(__int_as_float(en[u].y),
                            ex2_ftz(__fsub_rn(pp[u].x, c.ctH) + __fsub_rn(pp[u].y, c.ctR)), s[u]);
        }
        float ls[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            live[u] = s[u] > 0.0f;
            ls[u] = lg2_approx(s[u]);
        }
        if (KIND == 1) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                xfH[u] = __fadd_rn(xfH[u], c.ctH);
                xfL[u] = __fadd_rn(xfL[u], __fadd_rn(c.ctR, ls[u]));
            }
        } else {
            float4 k0[U], t0[U], t1[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const FallT &F = fall[R[u].meta >> 8];
                k0[u] = F.k0;
                t0[u] = F.t0;
                t1[u] = F.t1;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                float H0 = k0[u].x, L0 = fmaf(t0[u].x, c.d1h, k0[u].y);
                acc_prod(H0, L0, k0[u].z, k0[u].w, c.d2h, c.d2l);
                // log2 Pr = log2 k0 - log2 k_inf + log2 M
                const float pH = __fadd_rn(__fsub_rn(H0, xfH[u]), c.ctH);
                const float pL = __fadd_rn(__fadd_rn(__fsub_rn(L0, xfL[u]), c.ctR), ls[u]);
                const float lPr = pH + pL;
                // log2(Pr / (1 + Pr)) without cancellation on either side of Pr = 1
                const bool low = lPr < 0.0f;
                const float t1p = lg2_approx(1.0f + ex2_ftz(low ? lPr : -lPr));
                float fL = low ? __fsub_rn(pL, t1p) : -t1p;
                if (KIND == 3) {
                    // Troe broadening (Gilbert-Luther-Troe form), log10 F from log2 units
                    const float Fc = fmaf(t0[u].y, ex2_ftz(c.Tf * t0[u].w),
                                          fmaf(t0[u].z, ex2_ftz(c.Tf * t1[u].x),
                                               t1[u].z * ex2_ftz(t1[u].y * c.invT)));
                    const float lFc = lg2_approx(Fc) * 0.30102999566398120f;
                    const float c1 = -0.4f - 0.67f * lFc, nn = 0.75f - 1.27f * lFc;
                    const float xx = lPr * 0.30102999566398120f + c1;
                    const float f1 = __fdividef(xx, nn - 0.14f * xx);
                    fL = __fadd_rn(fL, __fdividef(lFc, 1.0f + f1 * f1) * 3.3219280948873623f);
                }
                xfH[u] = low ? __fadd_rn(xfH[u], pH) : xfH[u];
                xfL[u] = __fadd_rn(xfL[u], fL);
            }
        }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        xrH[u] = __fadd_rn(xfH[u], rb[u]);
        xrL[u] = xfL[u];
    }
    // species terms (heads exact on the grid)
#pragma unroll
    for (int t = 0; t < NF; ++t) {
        float4 P[U];
        float nu[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            int off;
            entry(R[u], rxnt_react(t), off, nu[u]);
            P[u] = load_pf(pfh, pfl, off);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            xfH[u] = fmaf(nu[u], P[u].x, xfH[u]);
            xfL[u] = fmaf(nu[u], P[u].y, xfL[u]);
            xrH[u] = fmaf(nu[u], P[u].z, xrH[u]);
            xrL[u] = fmaf(nu[u], P[u].w, xrL[u]);
        }
    }
#pragma unroll
    for (int t = 0; t < NR; ++t) {
        float4 P[U];
        float nu[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            int off;
            entry(R[u], rxnt_prod(t), off, nu[u]);
            P[u] = load_pf(pfh, pfl, off);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            xrH[u] = fmaf(nu[u], __fsub_rn(P[u].x, P[u].z), xrH[u]);
            xrL[u] = fmaf(nu[u], __fsub_rn(P[u].y, P[u].w), xrL[u]);
        }
    }
    float q[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        // 2^(H + L) as 2^H 2^L: H is exact, so the exponent is never rounded at its own
        // magnitude
        const float qn = ex2_ftz(xfH[u]) * ex2_ftz(xfL[u]) - ex2_ftz(xrH[u]) * ex2_ftz(xrL[u]);
        q[u] = live[u] ? qn : 0.0f;
    }
#pragma unroll
    for (int g = 0; g < U; g += kQuad) scatter_quad<NN>(R + g, om, q + g);
}

__device__ __forceinline__ void copy16(void *dst, const void *src, size_t bytes)
{
    for (size_t o = threadIdx.x * 16; o < bytes; o += (size_t)blockDim.x * 16)
        *(float4 *)((char *)dst + o) = __ldg((const float4 *)((const char *)src + o));
}

// log2 m for m in [0.5, 1): m' = m or 2 m in [0.75, 1.5), ln m' = 2 atanh(s) with
// s = (m' - 1) / (m' + 1), |s| <= 1/5, series to s^11 (truncation < 2e-10)
__device__ __forceinline__ float log2_mant(float m)
{
    const bool lo = m < 0.75f;
    const float mm = lo ? 2.0f * m : m;
    const float s = __fdividef(__fsub_rn(mm, 1.0f), __fadd_rn(mm, 1.0f));
    const float s2 = s * s;
    float t = fmaf(s2, 1.0f / 11.0f, 1.0f / 9.0f);
    t = fmaf(s2, t, 1.0f / 7.0f);
    t = fmaf(s2, t, 1.0f / 5.0f);
    t = fmaf(s2, t, 1.0f / 3.0f);
    return fmaf(2.0f * fmaf(s * s2, t, s), 1.4426950408889634f, lo ? -1.0f : 0.0f);
}

// U consecutive species of the lane's cell: z_k = Y_k / W_k into the double-float sum (in
// species order), P_k = log2 z_k as exact exponent + grid head of the mantissa's log2 (the
// cell's shift to log2 C_k is added later), F_k = G_k(T) + log2(p_ref/RT); out: P/F rows
template <int U>
__device__ __forceinline__ void species_block(const SpecT *sp, const float *yrow, int rg,
                                              const CellF &c, float d1l, float u, float gpH,
                                              float gpR, float &zh, float &zl, char *out_h,
                                              char *out_l)
{
    float4 ga[U], gb[U], gc[U];
    float z[U], Ph[U], Pl[U], FH[U], FL[U];
#pragma unroll
    for (int v = 0; v < U; ++v) {
        ga[v] = sp[v].ga[rg];
        gb[v] = sp[v].gb[rg];
        gc[v] = sp[v].gc[rg];
    }
#pragma unroll
    for (int v = 0; v < U; ++v) z[v] = fmaxf(yrow[v], 0.0f) * gc[v].z;
#pragma unroll
    for (int v = 0; v < U; ++v) {                // two-sum into (zh, zl), species order
        const float s = __fadd_rn(zh, z[v]), bb = __fsub_rn(s, zh);
        zl = __fadd_rn(zl, __fadd_rn(__fsub_rn(zh, __fsub_rn(s, bb)), __fsub_rn(z[v], bb)));
        zh = s;
    }
#pragma unroll
    for (int v = 0; v < U; ++v) {
        // z = m 2^ex, m in [0.5, 1) (subnormal z scaled by 2^24 first)
        const bool sub = z[v] < 1.17549435e-38f;
        const int bits = __float_as_int(sub ? z[v] * 16777216.0f : z[v]);
        const int ex = ((bits >> 23) & 0xFF) - 126 - (sub ? 24 : 0);
        const float lm = log2_mant(__int_as_float((bits & 0x007FFFFF) | 0x3F000000));
        const float lmh = grid12(lm);
        Ph[v] = z[v] > 0.0f ? __fadd_rn((float)ex, lmh) : kAbsentLog2;
        Pl[v] = z[v] > 0.0f ? __fsub_rn(lm, lmh) : 0.0f;
    }
#pragma unroll
    for (int v = 0; v < U; ++v) {
        FH[v] = __fadd_rn(ga[v].x, gpH);
        FL[v] = __fadd_rn(ga[v].y, gpR);
    }
#pragma unroll
    for (int v = 0; v < U; ++v) acc_prod(FH[v], FL[v], ga[v].z, ga[v].w, c.d1h, d1l);
#pragma unroll
    for (int v = 0; v < U; ++v) acc_prod(FH[v], FL[v], gb[v].x, gb[v].y, c.d2h, c.d2l);
#pragma unroll
    for (int v = 0; v < U; ++v)
        FL[v] = __fadd_rn(FL[v], u * fmaf(u, fmaf(u, fmaf(u, gc[v].y, gc[v].x), gb[v].w), gb[v].z));
#pragma unroll
    for (int v = 0; v < U; ++v) {
        // F's remainder back under 2^-12 (its polynomial part is not small), for FP16
        const float fh = grid12(FL[v]);
        *(float2 *)(out_h + v * kPfRow) = make_float2(Ph[v], __fadd_rn(FH[v], fh));
        *(__half2 *)(out_l + v * kPfRow) = __floats2half2_rn(Pl[v], __fsub_rn(FL[v], fh));
    }
}

constexpr int kMaxWarps = 8;
constexpr int kPieces = kChunk * (int)sizeof(RxnT) / 16;          // float4 pieces per chunk

__global__ void __launch_bounds__(32 * kMaxWarps, 1)
k_source_f32t(F32TView v, int64_t n, const float *__restrict__ T, const float *__restrict__ P,
              const float *__restrict__ Y, int64_t ldY, float *__restrict__ om, int64_t ldO)
{
    extern __shared__ __align__(16) unsigned char s_raw[];
    const int ns = v.ns, lane = threadIdx.x & 31, w = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    // block tables
    SpecT *s_spec = (SpecT *)s_raw;
    size_t off = a16(sizeof(SpecT) * ns);
    int2 *s_tb = (int2 *)(s_raw + off);
    off += a16(sizeof(int2) * v.n_tb);
    FallT *s_fall = (FallT *)(s_raw + off);
    off += a16(sizeof(FallT) * v.n_fall);
    RxnT *s_rec = (RxnT *)(s_raw + off);
    off += 2 * kChunk * sizeof(RxnT);
    unsigned char *wbase = s_raw + off + (size_t)w * (warp_pf_bytes(ns) + warp_om_bytes(ns));
    char *pfh_w = (char *)wbase + lane * 8;                   // this lane's P/F columns
    char *pfl_w = (char *)wbase + kPfHead + lane * 4;
    float *s_om = (float *)(wbase + warp_pf_bytes(ns));
    copy16(s_spec, v.spec, sizeof(SpecT) * ns);
    for (int t = threadIdx.x; t < v.n_tb; t += blockDim.x) s_tb[t] = __ldg(v.tb + t);
    copy16(s_fall, v.fall, sizeof(FallT) * v.n_fall);
    copy16(s_rec, v.rxn, sizeof(RxnT) * kChunk);
    __syncthreads();

    // the warp's cells; a warp past the batch redoes the last cell and stores nothing
    const int64_t i0 = ((int64_t)blockIdx.x * wpb + w) * 32;
    const int nc = i0 < n ? (int)(n - i0 < 32 ? n - i0 : 32) : 0;
    const int64_t ib = i0 < n ? i0 : n - 1;
    const int ncl = nc > 0 ? nc : 1;
    const int me = lane < ncl ? lane : ncl - 1;
    const int64_t i = ib + me;

    // ---- per-cell features in double-float arithmetic
    CellF c;
    c.Tf = T[i];
    const dflt log2e = df_of(v.log2e);
    const dflt lT = df_log2f(c.Tf, log2e);
    const dflt d1 = df_add(lT, df_neg(df_of(v.lg2T0)));                 // log2 T - log2 T0
    c.d1h = d1.h;
    const float d1l = d1.l;
    c.invT = __fdiv_rn(1.0f, c.Tf);
    const dflt rT = {c.invT, __fmul_rn(c.invT, fmaf(-c.Tf, c.invT, 1.0f))};   // 1/T
    const dflt d2 = df_add(rT, df_neg(df_of(v.invT0)));                 // 1/T - 1/T0
    c.d2h = d2.h;
    c.d2l = d2.l;
    const int rg = (double)c.Tf >= v.t_mid ? 1 : 0;
    const float u = __fmul_rn(__fsub_rn(c.Tf, v.Tc[rg]), 1e-3f);        // (T - T_c) / 1000
    // log2 c_tot = log2(P / (R T)); log2(p_ref / (R T))
    grid_split(df_add(df_add(df_log2f(P[i], log2e), df_neg(df_of(v.lg2R))), df_neg(lT)), c.ctH, c.ctR);
    float gpH, gpR;
    grid_split(df_add(df_of(v.lg2_pref_R), df_neg(lT)), gpH, gpR);

    // ---- species: z_k = Y_k / W_k, log2 z_k (exact exponent + grid head of the mantissa's
    // log2), sum_k z_k (double-float), F_k; Y staged 32 species at a time (coalesced rows)
    float zh = 0.0f, zl = 0.0f;
    for (int k0 = 0; k0 < ns; k0 += 32) {
        const int kn = ns - k0 < 32 ? ns - k0 : 32;
        __syncwarp();
        if (lane < kn)
            for (int cc = 0; cc < ncl; ++cc) s_om[cc * kOmStride + lane] = Y[(ib + cc) * ldY + k0 + lane];
        __syncwarp();
        const float *yrow = s_om + me * kOmStride;
        int kk = 0;
        for (; kk + kQuad <= kn; kk += kQuad)
            species_block<kQuad>(s_spec + k0 + kk, yrow + kk, rg, c, d1l, u, gpH, gpR, zh, zl,
                                 pfh_w + (k0 + kk) * kPfRow, pfl_w + (k0 + kk) * kPfRow);
        for (; kk < kn; ++kk)
            species_block<1>(s_spec + k0 + kk, yrow + kk, rg, c, d1l, u, gpH, gpR, zh, zl,
                             pfh_w + (k0 + kk) * kPfRow, pfl_w + (k0 + kk) * kPfRow);
    }
    // log2 C_k = log2 z_k + log2(c_tot / sum z): add the cell's shift to every P_k
    float cnH = c.ctH, cnR = c.ctR;
    if (zh > 0.0f) {
        const dflt ls = df_log2f(zh, log2e);
        float lsH, lsR;
        grid_split({ls.h, __fadd_rn(ls.l, __fmul_rn(__fdiv_rn(zl, zh), log2e.h))}, lsH, lsR);
        cnH = __fsub_rn(cnH, lsH);
        cnR = __fsub_rn(cnR, lsR);
    }
    __syncwarp();
    for (int k = 0; k < ns; ++k) {
        float *ph = (float *)(pfh_w + k * kPfRow);
        __half2 *pl = (__half2 *)(pfl_w + k * kPfRow);
        *ph = __fadd_rn(*ph, cnH);
        const float2 l = __half22float2(*pl);
        *pl = __floats2half2_rn(__fadd_rn(l.x, cnR), l.y);
        s_om[k * kOmStride + lane] = 0.0f;
    }
    *(float2 *)(pfh_w + ns * kPfRow) = make_float2(0.0f, 0.0f);       // the zero row
    *(__half2 *)(pfl_w + ns * kPfRow) = __floats2half2_rn(0.0f, 0.0f);
    s_om[ns * kOmStride + lane] = 0.0f;

    // ---- reactions: chunks of records staged one ahead, quads of one group type
    const char *pfh = pfh_w, *pfl = pfl_w;
    char *omc = (char *)s_om + lane * 4;
    const int nch = v.n_rec / kChunk;
    const float4 *src = (const float4 *)v.rxn;
    for (int ch = 0; ch < nch; ++ch) {
        float4 pre[kPieces / 32];
        const bool more = ch + 1 < nch;
        if (more) {
#pragma unroll
            for (int r = 0; r < kPieces / 32; ++r) {
                const int p = threadIdx.x + r * blockDim.x;
                if (p < kPieces) pre[r] = __ldg(src + (size_t)(ch + 1) * kPieces + p);
            }
        }
        const RxnT *rc = s_rec + (ch & 1) * kChunk;
#pragma unroll 1
        for (int r = 0; r < kChunk;) {
            const RxnT *R = rc + r;
            const uint32_t ty = R->meta & 7u;
            // two elementary quads of one type: eight rate chains at once, two omega rounds
            if (ty <= kGBig && r + 2 * kQuad <= kChunk && (R[kQuad].meta & 7u) == ty) {
                if (ty == kGSmall)
                    quad<2, 2, 4, 0, 2 * kQuad>(R, pfh, pfl, omc, s_tb, s_fall, c);
                else
                    quad<3, 3, 6, 0, 2 * kQuad>(R, pfh, pfl, omc, s_tb, s_fall, c);
                r += 2 * kQuad;
                continue;
            }
            switch (ty) {
            case kGSmall: quad<2, 2, 4, 0>(R, pfh, pfl, omc, s_tb, s_fall, c); break;
            case kGBig: quad<3, 3, 6, 0>(R, pfh, pfl, omc, s_tb, s_fall, c); break;
            case kGThird: quad<3, 3, 6, 1>(R, pfh, pfl, omc, s_tb, s_fall, c); break;
            case kGLind: quad<3, 3, 6, 2>(R, pfh, pfl, omc, s_tb, s_fall, c); break;
            default: quad<3, 3, 6, 3>(R, pfh, pfl, omc, s_tb, s_fall, c); break;
            }
            r += kQuad;
        }
        if (more) {
            float4 *dst = (float4 *)(s_rec + ((ch + 1) & 1) * kChunk);
#pragma unroll
            for (int r = 0; r < kPieces / 32; ++r) {
                const int p = threadIdx.x + r * blockDim.x;
                if (p < kPieces) dst[p] = pre[r];
            }
        }
        __syncthreads();
    }

    // ---- omega rows out, lanes over species
    __syncwarp();
    for (int cc = 0; cc < nc; ++cc)
        for (int k = lane; k < ns; k += 32) om[(i0 + cc) * ldO + k] = s_om[k * kOmStride + cc];
}

}  // namespace

chem_status launch_source_fp32_t(const chem_mech *m, int64_t n, const float *T, const float *P,
                                 const float *Y, int64_t ldY, float *om, int64_t ldO,
                                 cudaStream_t s)
{
    static SmemOptIn opt;
    static std::atomic<int> sm_count[64];       // per device index (chem_source_term checks < 64)
    if (n <= 0) return CHEM_OK;
    if (!m->vt.ok) return set_error(CHEM_EUNSUPPORTED, "fp32: no thread-per-cell tables");
    int dev = 0;
    cudaGetDevice(&dev);
    int nsm = dev >= 0 && dev < 64 ? sm_count[dev].load(std::memory_order_relaxed) : 0;
    if (nsm <= 0) {
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (nsm <= 0) nsm = 1;
        if (dev >= 0 && dev < 64) sm_count[dev].store(nsm, std::memory_order_relaxed);
    }
    const size_t fixed = block_fixed_bytes(m->vt), per_warp = warp_pf_bytes(m->ns) + warp_om_bytes(m->ns);
    if (fixed + per_warp > kTSmemMax)          // excluded when the tables were built
        return set_error(CHEM_EUNSUPPORTED, "fp32: thread-per-cell tables exceed shared memory");
    int wmax = (int)((kTSmemMax - fixed) / per_warp);
    wmax = wmax < 1 ? 1 : wmax > kMaxWarps ? kMaxWarps : wmax;
    // warps per block: enough blocks to cover every SM before blocks grow
    const int64_t warps = (n + 31) / 32;
    int64_t wpb = (warps + nsm - 1) / nsm;
    wpb = wpb < 1 ? 1 : wpb > wmax ? wmax : wpb;
    const int64_t blocks = (warps + wpb - 1) / wpb;
    const size_t smem = fixed + (size_t)wpb * per_warp;
    chem_status st = launch_opted(opt, (const void *)k_source_f32t, (int)kTSmemMax, "fp32", [&] {
        k_source_f32t<<<(unsigned)blocks, (unsigned)(32 * wpb), smem, s>>>(m->vt, n, T, P, Y, ldY, om, ldO);
    });
    if (st == CHEM_OK) g_launches.fetch_add(1);
    return st;
}

}  // namespace chem
