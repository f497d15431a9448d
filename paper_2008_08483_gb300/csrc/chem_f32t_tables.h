// chem_f32t_tables.h -- host-side tables of the thread-per-cell FP32 source-term kernel
// (kern_f32t.cu), built from the mechanism descriptor: the reaction records in the kernel's
// processing order (type groups, quads from chem_quads.h, zero-rate padding), the centred
// Gibbs records of the species, the quads' interleaved third-body efficiency lists and the
// falloff records, with the double-float constants of the per-cell features.  Host code
// only; kern_f32t.cu uploads the tables and tests/f32t_tables_driver.cpp checks them.
#pragma once

#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "chem_internal.h"
#include "chem_quads.h"

namespace chem {
namespace f32t {

constexpr int kTMaxSpecies = 192;
constexpr double kT0 = 1000.0;               // centre of the temperature features (K)
constexpr float kGridAdd = 3072.0f;          // 1.5 * 2^11: (x + it) - it rounds x to 2^-12
                                             // for |x| < 2^10
constexpr double kGridLimit = 1024.0;        // |head| of a table value (exact sums to 2^11)
constexpr float kAbsentLog2 = -1000.0f;      // log2 C of an absent species (2^x flushes to 0)
constexpr float kOff = -2000.0f;             // exponent bias of padding and irreversible rates
constexpr int kChunk = 16;                   // reaction records per staged chunk
constexpr int kOmStride = 33;                // omega tile row (odd: conflict-free both ways)
// one species row of the P/F table: 32 lanes of (P_h, F_h) as float2, then 32 lanes of
// (P_l, F_l) as half2 (remainders below 2^-12: FP16 keeps them to ~6e-8)
constexpr int kPfHead = 32 * 8;
constexpr int kPfRow = kPfHead + 32 * 4;
constexpr int kOmRow = kOmStride * 4;        // bytes of one omega tile row
// group types, in processing order
enum { kGSmall = 0, kGBig = 1, kGThird = 2, kGLind = 3, kGTroe = 4, kGroups = 5 };

inline double grid_head(double x) { return rint(x * 4096.0) / 4096.0; }

// (hi, lo) float pair of a double
inline void dsplit2(double x, float &h, float &l)
{
    h = (float)x;
    l = (float)(x - (double)h);
}

constexpr int kQuad = 4;                     // reactions taken together (groups padded to it)

inline void put_entry(RxnT &r, int pair, int off, float nu)
{
    r.ent[2 * pair] = off;
    memcpy(&r.ent[2 * pair + 1], &nu, 4);
}
// every entry at the zero row with coefficient 0
inline void clear_entries(RxnT &r, int ns)
{
    for (int s = 0; s < kTSide; ++s) {
        put_entry(r, rxnt_react(s), ns * kPfRow, 0.0f);
        put_entry(r, rxnt_prod(s), ns * kPfRow, 0.0f);
    }
    for (int s = 0; s < kTNet; ++s) put_entry(r, rxnt_net(s), ns * kOmRow, 0.0f);
}

// log2 k(T) = log2 k(T0) + b d1 - (E/R) log2 e d2 (Eq. 6) as (H, L, coefficient of d2)
inline bool centred(const double *a, float4 &out, float &b)
{
    const double at0 = (a[0] + a[1] * log(kT0) - a[2] / kT0) * kLog2e;
    const double h = grid_head(at0);
    if (!(fabs(h) < kGridLimit)) return false;
    float th, tl;
    dsplit2(-a[2] * kLog2e, th, tl);
    out = make_float4((float)h, (float)(at0 - h), th, tl);
    b = (float)a[1];
    return true;
}

__host__ __device__ inline size_t a16(size_t x) { return (x + 15) & ~(size_t)15; }
// shared memory of one warp: P/F rows (+ the zero row of unused entries) and the omega tile
// (at least 32 rows: it first stages the Y rows of the warp's cells)
__host__ __device__ inline size_t warp_pf_bytes(int ns) { return (size_t)(ns + 1) * kPfRow; }
__host__ __device__ inline size_t warp_om_bytes(int ns)
{
    return a16((size_t)(ns + 1 > 32 ? ns + 1 : 32) * kOmRow);
}
// shared memory of the block's staged tables: species, third-body lists, falloff, two chunks
__host__ __device__ inline size_t block_fixed_bytes(const F32TView &v)
{
    return a16(sizeof(SpecT) * v.ns) + a16(sizeof(int2) * v.n_tb) + a16(sizeof(FallT) * v.n_fall) +
           2 * kChunk * sizeof(RxnT);
}
constexpr size_t kTSmemMax = 227 * 1024;       // dynamic shared memory of one block


struct Tables {
    std::vector<RxnT> rx;          // records, processing order, a multiple of kChunk
    std::vector<int> order;        // reaction of each record, -1 for a padding record
    std::vector<SpecT> sp;
    std::vector<int2> tb;          // (row offset, efficiency - 1 as float bits)
    std::vector<FallT> fall;
    F32TView v;                    // sizes and constants (device pointers unset, ok false)
};

// The tables of a mechanism; false when it is outside the kernel's limits (above kTMaxSpecies
// species, more than three species a side, heads beyond the exact range, or tables beyond
// shared memory): the FP32 source term then runs the warp-per-cell kernel.
inline bool build_tables(const chem_mech_desc *d, Tables &t)
{
    const int ns = d->n_species, nr = d->n_reactions;
    if (ns > kTMaxSpecies) return false;
    std::vector<RxnT> rx;
    std::vector<int> order;
    std::vector<int> type_of(nr);
    std::vector<int2> tb;
    std::vector<FallT> fall;
    std::vector<RxnT> one(nr);
    std::vector<std::vector<int2>> lists(nr);      // listed efficiencies (row offset, eff - 1)
    for (int j = 0; j < nr; ++j) {
        RxnT &r = one[j];
        memset(&r, 0, sizeof r);
        if (!centred(d->arrh + (size_t)j * 3, r.kf, r.b)) return false;
        const int kind = d->kind[j];
        int nf = 0, nrr = 0, nnet = 0;
        clear_entries(r, ns);
        for (int k = 0; k < ns; ++k) {
            const int f = d->nu_f[(size_t)j * ns + k], p = d->nu_r[(size_t)j * ns + k];
            if (f) {
                if (nf >= kTSide) return false;
                put_entry(r, rxnt_react(nf++), k * kPfRow, (float)f);
            }
            if (p) {
                if (nrr >= kTSide) return false;
                put_entry(r, rxnt_prod(nrr++), k * kPfRow, (float)p);
            }
            if (p != f) {
                if (nnet >= kTNet) return false;
                put_entry(r, rxnt_net(nnet++), k * kOmRow, (float)(p - f));
            }
        }
        r.rb = d->reversible[j] ? 0.0f : kOff;
        const int type = kind == 0 ? (nf <= 2 && nrr <= 2 && nnet <= 4 ? kGSmall : kGBig)
                                   : kind == 1 ? kGThird : kind == 2 ? kGLind : kGTroe;
        type_of[j] = type;
        uint32_t fidx = 0;
        if (kind >= 2) {
            FallT f;
            memset(&f, 0, sizeof f);
            float b0;
            if (!centred(d->arrh_low + (size_t)j * 3, f.k0, b0)) return false;
            f.t0.x = b0;
            if (kind == 3) {
                const double *t = d->troe + (size_t)j * 4;
                // F_cent = (1 - alpha) 2^(T t0.w) + alpha 2^(T t1.x) + t1.z 2^(t1.y / T)
                f.t0.y = (float)(1.0 - t[0]);
                f.t0.z = (float)t[0];
                f.t0.w = (float)(-kLog2e / t[1]);
                f.t1.x = (float)(-kLog2e / t[2]);
                f.t1.y = t[3] > 0.0 ? (float)(-t[3] * kLog2e) : 0.0f;
                f.t1.z = t[3] > 0.0 ? 1.0f : 0.0f;
            }
            fidx = (uint32_t)fall.size();
            fall.push_back(f);
        }
        r.meta = (uint32_t)type | (fidx << 8);
        if (kind >= 1)
            for (int k = 0; k < ns; ++k) {
                const double e = d->eff ? d->eff[(size_t)j * ns + k] : 1.0;
                if (e != 1.0) {
                    const float ef = (float)(e - 1.0);
                    int bits;
                    memcpy(&bits, &ef, 4);
                    lists[j].push_back(make_int2(k * kPfRow, bits));
                }
            }
    }
    // records in quads of one type, net species pairwise distinct where the greedy packing
    // allows (chem_quads.h; meta bit 3: one omega round trip), zero-rate padding records
    std::vector<std::vector<int>> net(nr);
    for (int j = 0; j < nr; ++j)
        for (int k = 0; k < ns; ++k)
            if (d->nu_r[(size_t)j * ns + k] != d->nu_f[(size_t)j * ns + k]) net[j].push_back(k);
    const QuadPlan plan = plan_quads(kGroups, type_of, net, kQuad);
    for (size_t qn = 0; qn < plan.type.size(); ++qn) {
        const size_t first = rx.size();
        const int *js = &plan.slot[qn * kQuad];
        size_t nit = 0;
        for (int u = 0; u < kQuad; ++u) {
            order.push_back(js[u]);
            if (js[u] >= 0) {
                rx.push_back(one[js[u]]);
                nit = std::max(nit, lists[js[u]].size());
            } else {
                RxnT pad = rx.back();                  // same type, zero rate
                pad.kf = make_float4(kOff, 0.0f, 0.0f, 0.0f);
                pad.b = 0.0f;
                clear_entries(pad, ns);
                rx.push_back(pad);
            }
        }
        // the quad's efficiency lists as [entry][reaction], padded with zero entries
        if (tb.size() + nit * kQuad > 65535 || nit > 65535) return false;
        const size_t base = tb.size();
        for (size_t it = 0; it < nit; ++it)
            for (int u = 0; u < kQuad; ++u) {
                const bool real = js[u] >= 0 && it < lists[js[u]].size();
                tb.push_back(real ? lists[js[u]][it] : make_int2(ns * kPfRow, 0));
            }
        rx[first].tb = (uint32_t)base | ((uint32_t)nit << 16);
        if (plan.disjoint[qn]) rx[first].meta |= 8u;
    }
    while (rx.size() % kChunk) {
        RxnT pad;
        memset(&pad, 0, sizeof pad);
        pad.kf = make_float4(kOff, 0.0f, 0.0f, 0.0f);
        pad.meta = kGSmall;
        clear_entries(pad, ns);
        rx.push_back(pad);
        order.push_back(-1);
    }
    // Gibbs layer per species and T range (Eq. 10 with NASA-7 a0..a6):
    //   G(T) = -g/(RT) log2 e = a0 log2 T + log2 e (a6 - a0 + a1 T/2 + a2 T^2/6 + a3 T^3/12
    //          + a4 T^4/20 - a5 / T)
    //        = G_c + a0 d1 - a5 log2 e d2 + sum_p e_p u^p,  u = (T - T_c) / 1000,
    // d1 and d2 centred on T0 as for the Arrhenius terms, the powers of T re-expanded about
    // the range's own centre T_c (0.65 and 2.25 t_mid: |u| <= 1.25 up to 3.5 t_mid), and the
    // constant of that expansion collected in G_c
    std::vector<SpecT> sp(ns);
    const double lg2T0 = log2(kT0);
    const double Tc[2] = {rint(0.65 * d->t_mid), rint(2.25 * d->t_mid)};
    static const double binom[5][5] = {{1, 0, 0, 0, 0}, {1, 1, 0, 0, 0}, {1, 2, 1, 0, 0},
                                       {1, 3, 3, 1, 0}, {1, 4, 6, 4, 1}};
    for (int k = 0; k < ns; ++k) {
        SpecT &s = sp[k];
        memset(&s, 0, sizeof s);
        for (int rg = 0; rg < 2; ++rg) {
            const double *a = d->nasa7 + (size_t)k * 14 + (size_t)rg * 7;
            const double c[5] = {0.0, a[1] / 2.0 * 1e3, a[2] / 6.0 * 1e6, a[3] / 12.0 * 1e9,
                                 a[4] / 20.0 * 1e12};        // on tau^m, tau = T / 1000
            // sum_m c_m (tau^m - 1) with tau = tc + u: the constant sum_m c_m (tc^m - 1), and
            // e_p = sum_{m >= p} C(m, p) c_m tc^(m - p) on u^p (binomial expansion)
            const double tc = Tc[rg] / 1000.0;
            double e[5] = {0.0, 0.0, 0.0, 0.0, 0.0}, cst = 0.0;
            for (int m = 1; m <= 4; ++m) {
                cst += c[m] * (pow(tc, m) - 1.0);
                for (int q = 1; q <= m; ++q) e[q] += binom[m][q] * c[m] * pow(tc, m - q);
            }
            const double g0 = a[0] * lg2T0 + kLog2e * (a[6] - a[0] + c[1] + c[2] + c[3] + c[4] -
                                                       a[5] / kT0 + cst);
            const double h = grid_head(g0);
            if (!(fabs(h) < kGridLimit)) return false;
            const double e1 = e[1], e2 = e[2], e3 = e[3], e4 = e[4];
            float a0h, a0l, a5h, a5l;
            dsplit2(a[0], a0h, a0l);
            dsplit2(-a[5] * kLog2e, a5h, a5l);
            s.ga[rg] = make_float4((float)h, (float)(g0 - h), a0h, a0l);
            s.gb[rg] = make_float4(a5h, a5l, (float)(e1 * kLog2e), (float)(e2 * kLog2e));
            s.gc[rg] = make_float4((float)(e3 * kLog2e), (float)(e4 * kLog2e),
                                   (float)(1.0 / d->mol_weight[k]), 0.0f);
        }
    }
    F32TView &v = t.v;
    v = F32TView{};
    v.ns = ns;
    v.n_rec = (int)rx.size();
    v.n_tb = (int)tb.size();
    v.n_fall = (int)fall.size();
    v.t_mid = d->t_mid;
    auto df2c = [](double x) {
        float h, l;
        dsplit2(x, h, l);
        return make_float2(h, l);
    };
    v.lg2T0 = df2c(log2(kT0));
    v.invT0 = df2c(1.0 / kT0);
    v.lg2R = df2c(log2(kR));
    v.lg2_pref_R = df2c(log2(d->p_ref / kR));
    v.log2e = df2c(kLog2e);
    v.Tc[0] = (float)Tc[0];
    v.Tc[1] = (float)Tc[1];
    // the kernel needs one warp's tables and the block's staged tables in shared memory
    if (block_fixed_bytes(v) + warp_pf_bytes(ns) + warp_om_bytes(ns) > kTSmemMax) return false;
    v.ok = false;
    t.rx = std::move(rx);
    t.order = std::move(order);
    t.sp = std::move(sp);
    t.tb = std::move(tb);
    t.fall = std::move(fall);
    return true;
}

}  // namespace f32t
}  // namespace chem
