// chem_mech.cu -- mechanism validation, load-time preprocessing and device upload.
//
// Load-time work (all in double precision on the host):
//  * sparse per-reaction species lists for the SIMT paths;
//  * the Arrhenius layer coefficients (Eq. 6) in natural-log (FP64 path) and log2
//    double-float (FP32 path) form;
//  * the Gibbs layer (Eq. 10) folded through the net stoichiometry (Eq. 11): the
//    coefficients of ln K_c on [1, ln T, tau, ..., tau^4, 1/T] per temperature range,
//    where the species cancellation of sum_k nu_kj g_k happens in double precision;
//  * third-body efficiency lists (efficiency - 1 for the species that differ from 1,
//    since M = sum_k eff_k C_k = c_tot + sum_k (eff_k - 1) C_k, Sec. 2.4).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "chem_internal.h"

namespace chem {

std::atomic<uint64_t> g_launches{0};
thread_local int tl_sm_limit = 0;

static thread_local std::string t_err;

chem_status set_error(chem_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_err = buf;
    return st;
}

void clear_error() { t_err.clear(); }

const char *last_error() { return t_err.c_str(); }

static float2 dsplit(double x)
{
    float h = (float)x;
    float l = (float)(x - (double)h);
    return make_float2(h, l);
}

void bf16_free_tables(chem_mech *m);
chem_status bf16_build_tables(chem_mech *m, const chem_mech_desc *d);

}  // namespace chem

using namespace chem;

extern "C" int32_t chem_abi_version(void) { return CHEM_ABI_VERSION; }

extern "C" const char *chem_last_error(void) { return chem::last_error(); }

extern "C" uint64_t chem_kernel_launch_count(void) { return g_launches.load(); }

static chem_status validate(const chem_mech_desc *d)
{
    if (!d) return set_error(CHEM_EINVAL, "descriptor is NULL");
    const int ns = d->n_species, nr = d->n_reactions;
    if (ns < 1 || ns > kMaxSpecies)
        return set_error(CHEM_EINVAL, "n_species=%d outside [1, %d]", ns, kMaxSpecies);
    if (nr < 1 || nr > kMaxReactions)
        return set_error(CHEM_EINVAL, "n_reactions=%d outside [1, %d]", nr, kMaxReactions);
    if (d->n_elements < 0) return set_error(CHEM_EINVAL, "n_elements < 0");
    if (!d->mol_weight || !d->nu_f || !d->nu_r || !d->arrh || !d->kind || !d->reversible ||
        !d->nasa7)
        return set_error(CHEM_EINVAL, "required descriptor array is NULL");
    if (d->n_elements > 0 && !d->elem_comp)
        return set_error(CHEM_EINVAL, "n_elements > 0 but elem_comp is NULL");
    if (!(d->t_mid > 0.0) || !isfinite(d->t_mid)) return set_error(CHEM_EINVAL, "t_mid must be > 0");
    if (!(d->p_ref > 0.0) || !isfinite(d->p_ref)) return set_error(CHEM_EINVAL, "p_ref must be > 0");
    for (int k = 0; k < ns; ++k) {
        if (!(d->mol_weight[k] > 0.0) || !isfinite(d->mol_weight[k]))
            return set_error(CHEM_EINVAL, "mol_weight[%d] must be finite and > 0", k);
        for (int c = 0; c < 14; ++c)
            if (!isfinite(d->nasa7[(size_t)k * 14 + c]))
                return set_error(CHEM_EINVAL, "nasa7 of species %d is not finite", k);
    }
    for (int j = 0; j < nr; ++j) {
        int nfs = 0, nrs = 0;
        for (int k = 0; k < ns; ++k) {
            int a = d->nu_f[(size_t)j * ns + k], b = d->nu_r[(size_t)j * ns + k];
            if (a < 0 || a > 127 || b < 0 || b > 127)
                return set_error(CHEM_EINVAL, "reaction %d: coefficient outside [0, 127]", j);
            nfs += a > 0;
            nrs += b > 0;
        }
        if (nfs < 1 || nrs < 1)
            return set_error(CHEM_EINVAL, "reaction %d: needs at least one reactant and product", j);
        if (nfs > kMaxSide || nrs > kMaxSide)
            return set_error(CHEM_EINVAL, "reaction %d: more than %d species on a side", j,
                             kMaxSide);
        for (int c = 0; c < 3; ++c)
            if (!isfinite(d->arrh[(size_t)j * 3 + c]))
                return set_error(CHEM_EINVAL, "reaction %d: Arrhenius parameters not finite", j);
        int kd = d->kind[j];
        if (kd < 0 || kd > 3) return set_error(CHEM_EINVAL, "reaction %d: kind %d", j, kd);
        if (d->reversible[j] != 0 && d->reversible[j] != 1)
            return set_error(CHEM_EINVAL, "reaction %d: reversible must be 0 or 1", j);
        if (kd >= 1 && d->eff) {
            for (int k = 0; k < ns; ++k) {
                double e = d->eff[(size_t)j * ns + k];
                if (!isfinite(e) || e < 0.0)
                    return set_error(CHEM_EINVAL, "reaction %d: efficiency must be finite, >= 0", j);
            }
        }
        if (kd >= 2) {
            if (!d->arrh_low)
                return set_error(CHEM_EINVAL, "reaction %d: falloff without arrh_low", j);
            for (int c = 0; c < 3; ++c)
                if (!isfinite(d->arrh_low[(size_t)j * 3 + c]))
                    return set_error(CHEM_EINVAL, "reaction %d: arrh_low not finite", j);
        }
        if (kd == 3) {
            if (!d->troe) return set_error(CHEM_EINVAL, "reaction %d: Troe without troe", j);
            const double *t = d->troe + (size_t)j * 4;
            if (!isfinite(t[0]) || !(t[1] > 0.0) || !(t[2] > 0.0) || !isfinite(t[1]) ||
                !isfinite(t[2]) || !isfinite(t[3]))
                return set_error(CHEM_EINVAL, "reaction %d: Troe needs finite alpha, T***>0, T*>0",
                                 j);
        }
        if (d->n_elements > 0) {
            for (int e = 0; e < d->n_elements; ++e) {
                long long bal = 0;
                for (int k = 0; k < ns; ++k) {
                    long long nu = (long long)d->nu_r[(size_t)j * ns + k] -
                                   d->nu_f[(size_t)j * ns + k];
                    bal += nu * d->elem_comp[(size_t)k * d->n_elements + e];
                }
                if (bal != 0)
                    return set_error(CHEM_EINVAL, "reaction %d is not balanced in element %d", j, e);
            }
        }
    }
    return CHEM_OK;
}

// ln K_c coefficients of reaction j, temperature range r, on [1, ln T, tau, tau^2, tau^3,
// tau^4, 1/T] (tau = T/1000).  With g/(RT) = a1 (1 - ln T) - a2 T/2 - a3 T^2/6 - a4 T^3/12
// - a5 T^4/20 + a6/T - a7 and ln K_c = -sum_k nu_k g_k/(RT) + dnu (ln(p_ref/R) - ln T).
namespace chem {
void fold_kc(const chem_mech_desc *d, int j, int r, double out[7])
{
    const int ns = d->n_species;
    double c[7] = {0, 0, 0, 0, 0, 0, 0};
    long dnu = 0;
    for (int k = 0; k < ns; ++k) {
        int nu = d->nu_r[(size_t)j * ns + k] - d->nu_f[(size_t)j * ns + k];
        if (!nu) continue;
        const double *a = d->nasa7 + (size_t)k * 14 + (size_t)r * 7;
        c[0] += -nu * (a[0] - a[6]);
        c[1] += nu * a[0];
        c[2] += nu * a[1] / 2.0 * 1e3;
        c[3] += nu * a[2] / 6.0 * 1e6;
        c[4] += nu * a[3] / 12.0 * 1e9;
        c[5] += nu * a[4] / 20.0 * 1e12;
        c[6] += -nu * a[5];
        dnu += nu;
    }
    c[0] += (double)dnu * log(d->p_ref / kR);
    c[1] -= (double)dnu;
    for (int m = 0; m < 7; ++m) out[m] = c[m];
}
}  // namespace chem

extern "C" chem_status chem_mechanism_load(const chem_mech_desc *d, chem_mech **out)
{
    clear_error();
    if (!out) return set_error(CHEM_EINVAL, "out is NULL");
    *out = nullptr;
    chem_status st = validate(d);
    if (st != CHEM_OK) return st;
    const int ns = d->n_species, nr = d->n_reactions;

    std::vector<RxnF64> r64(nr);
    std::vector<RxnF32> r32(nr);
    std::vector<SpecF32> s32(ns);
    std::vector<uint16_t> tb_sp;
    std::vector<double> tb_e64;
    std::vector<float> tb_e32;
    std::vector<double> invW(ns);
    for (int k = 0; k < ns; ++k) invW[k] = 1.0 / d->mol_weight[k];
    std::vector<RxnInt> rint(nr);
    bool int_ok = true;
    // integrator processing order: reactions grouped by kind, each kind padded to a multiple
    // of 32 slots so that a warp's 32 reactions share one kind
    std::vector<int32_t> order;
    for (int kd = 0; kd <= 3; ++kd) {
        for (int j = 0; j < nr; ++j)
            if (d->kind[j] == kd) order.push_back(j);
        while (order.size() % 32) order.push_back(-1);
    }

    for (int j = 0; j < nr; ++j) {
        RxnF64 &a = r64[j];
        RxnF32 &b = r32[j];
        memset(&a, 0, sizeof a);
        memset(&b, 0, sizeof b);
        const double *ar = d->arrh + (size_t)j * 3;
        a.lnA = ar[0];
        a.b = ar[1];
        a.EoR = ar[2];
        b.kf[0] = dsplit(ar[0] * kLog2e);
        b.kf[1] = dsplit(ar[1]);
        b.kf[2] = dsplit(-ar[2] * kLog2e);
        for (int r = 0; r < 2; ++r) fold_kc(d, j, r, a.kc[r]);
        a.kind = b.kind = d->kind[j];
        a.rev = b.rev = d->reversible[j];
        int nf = 0, nrr = 0, ordf = 0, ordr = 0;
        for (int k = 0; k < ns; ++k) {
            int f = d->nu_f[(size_t)j * ns + k], p = d->nu_r[(size_t)j * ns + k];
            if (f) {
                a.spf[nf] = b.spf[nf] = (uint16_t)k;
                a.nuf[nf] = b.nuf[nf] = (uint8_t)f;
                ++nf;
                ordf += f;
            }
            if (p) {
                a.spr[nrr] = b.spr[nrr] = (uint16_t)k;
                a.nur[nrr] = b.nur[nrr] = (uint8_t)p;
                ++nrr;
                ordr += p;
            }
        }
        a.nf = b.nf = nf;
        a.nr = b.nr = nrr;
        {
            RxnInt &c = rint[j];
            memset(&c, 0, sizeof c);
            for (int k = 0; k < ns && int_ok; ++k) {
                int f = d->nu_f[(size_t)j * ns + k], p = d->nu_r[(size_t)j * ns + k];
                if (!f && !p) continue;
                if (c.ncol >= kIntMax) {
                    int_ok = false;
                    break;
                }
                c.col_sp[c.ncol] = (uint16_t)k;
                c.col_nuf[c.ncol] = (uint8_t)f;
                c.col_nur[c.ncol] = (uint8_t)p;
                ++c.ncol;
                if (p != f) {
                    c.row_sp[c.nrow] = (uint16_t)k;
                    c.row_nu[c.nrow] = (double)(p - f);
                    ++c.nrow;
                }
            }
        }
        b.ordf = ordf;
        b.ordr = ordr;
        b.dnu = ordr - ordf;
        a.tb_begin = b.tb_begin = (int32_t)tb_sp.size();
        if (a.kind >= 1) {
            for (int k = 0; k < ns; ++k) {
                double e = d->eff ? d->eff[(size_t)j * ns + k] : 1.0;
                if (e != 1.0) {
                    tb_sp.push_back((uint16_t)k);
                    tb_e64.push_back(e - 1.0);
                    tb_e32.push_back((float)(e - 1.0));
                }
            }
        }
        a.tb_end = b.tb_end = (int32_t)tb_sp.size();
        if (a.kind >= 2) {
            const double *al = d->arrh_low + (size_t)j * 3;
            a.low[0] = al[0];
            a.low[1] = al[1];
            a.low[2] = al[2];
            b.k0[0] = dsplit(al[0] * kLog2e);
            b.k0[1] = dsplit(al[1]);
            b.k0[2] = dsplit(-al[2] * kLog2e);
        }
        if (a.kind == 3) {
            const double *t = d->troe + (size_t)j * 4;
            double tr[5] = {1.0 - t[0], t[0], 1.0 / t[1], 1.0 / t[2], t[3]};
            for (int c = 0; c < 5; ++c) {
                a.troe[c] = tr[c];
                b.troe[c] = (float)tr[c];
            }
        }
    }
    // FP32 Gibbs layer: -g_k/(RT) in log2 units on [1, log2 T, tau, tau^2, tau^3, tau^4, 1/T]
    for (int k = 0; k < ns; ++k) {
        memset(&s32[k], 0, sizeof s32[k]);
        s32[k].invW = (float)invW[k];
        for (int r = 0; r < 2; ++r) {
            const double *a = d->nasa7 + (size_t)k * 14 + (size_t)r * 7;
            double c[7] = {(-(a[0] - a[6])) * kLog2e, a[0], a[1] / 2.0 * 1e3 * kLog2e,
                           a[2] / 6.0 * 1e6 * kLog2e, a[3] / 12.0 * 1e9 * kLog2e,
                           a[4] / 20.0 * 1e12 * kLog2e, -a[5] * kLog2e};
            for (int m = 0; m < 7; ++m) s32[k].gl[r][m] = dsplit(c[m]);
        }
    }

    // one device blob
    auto align = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t o_r64 = 0;
    size_t o_s32 = align(o_r64 + sizeof(RxnF64) * nr);
    size_t o_tbsp = align(o_s32 + sizeof(SpecF32) * ns);
    size_t ntb = tb_sp.size() ? tb_sp.size() : 1;
    size_t o_tbe64 = align(o_tbsp + sizeof(uint16_t) * ntb);
    size_t o_tbe32 = align(o_tbe64 + sizeof(double) * ntb);
    size_t o_invw = align(o_tbe32 + sizeof(float) * ntb);
    size_t o_rint = align(o_invw + sizeof(double) * ns);
    size_t o_nasa = align(o_rint + sizeof(RxnInt) * nr);
    size_t o_w = align(o_nasa + sizeof(double) * 14 * ns);
    // per group of 32 slots: species -> (slot, net coefficient) lists
    const size_t n_groups = order.size() / 32;
    std::vector<int32_t> gptr(n_groups * (ns + 1) + 1, 0), gslot;
    std::vector<double> gnu;
    for (size_t g = 0; g < n_groups; ++g) {
        for (int k = 0; k < ns; ++k) {
            gptr[g * (ns + 1) + k] = (int32_t)gslot.size();
            for (int r = 0; r < 32; ++r) {
                int j = order[g * 32 + r];
                if (j < 0) continue;
                int nu = d->nu_r[(size_t)j * ns + k] - d->nu_f[(size_t)j * ns + k];
                if (nu) {
                    gslot.push_back(r);
                    gnu.push_back((double)nu);
                }
            }
        }
        gptr[g * (ns + 1) + ns] = (int32_t)gslot.size();
    }
    const size_t nge = gslot.size() ? gslot.size() : 1;
    // species-major net stoichiometry for the FP32 gather
    std::vector<int32_t> cptr(ns + 1, 0), crxn;
    std::vector<float> cnu;
    for (int k = 0; k < ns; ++k) {
        cptr[k] = (int32_t)crxn.size();
        for (int j = 0; j < nr; ++j) {
            const int nu = d->nu_r[(size_t)j * ns + k] - d->nu_f[(size_t)j * ns + k];
            if (nu) {
                crxn.push_back(j);
                cnu.push_back((float)nu);
            }
        }
    }
    cptr[ns] = (int32_t)crxn.size();
    const size_t nce = crxn.size() ? crxn.size() : 1;
    // species-major reaction sides (nu', nu'' of every reaction the species is on) and
    // listed third-body efficiencies (eff - 1), for the warp-per-cell vjp gather
    std::vector<int32_t> sdptr(ns + 1, 0), sdrxn, tsptr(ns + 1, 0), tsrxn;
    std::vector<float> sdnuf, sdnur;
    std::vector<double> tse;
    for (int k = 0; k < ns; ++k) {
        sdptr[k] = (int32_t)sdrxn.size();
        for (int j = 0; j < nr; ++j) {
            const int f = d->nu_f[(size_t)j * ns + k], r = d->nu_r[(size_t)j * ns + k];
            if (f || r) {
                sdrxn.push_back(j);
                sdnuf.push_back((float)f);
                sdnur.push_back((float)r);
            }
        }
        tsptr[k] = (int32_t)tsrxn.size();
        for (int j = 0; j < nr; ++j)
            for (int t = r64[j].tb_begin; t < r64[j].tb_end; ++t)
                if (tb_sp[t] == k) {
                    tsrxn.push_back(j);
                    tse.push_back(tb_e64[t]);
                }
    }
    sdptr[ns] = (int32_t)sdrxn.size();
    tsptr[ns] = (int32_t)tsrxn.size();
    const size_t nsd = sdrxn.size() ? sdrxn.size() : 1, nts = tsrxn.size() ? tsrxn.size() : 1;
    // species -> lanes for the gather: longest lists first, each to the least loaded lane
    std::vector<int32_t> lptr(33, 0), lsp;
    {
        std::vector<int> by(ns);
        for (int k = 0; k < ns; ++k) by[k] = k;
        std::stable_sort(by.begin(), by.end(), [&](int a, int b) {
            return cptr[a + 1] - cptr[a] > cptr[b + 1] - cptr[b];
        });
        std::vector<std::vector<int32_t>> lanes(32);
        std::vector<long> load(32, 0);
        for (int k : by) {
            int l = 0;
            for (int x = 1; x < 32; ++x)
                if (load[x] < load[l]) l = x;
            lanes[l].push_back(k);
            load[l] += 1 + (cptr[k + 1] - cptr[k]);
        }
        for (int l = 0; l < 32; ++l) {
            lptr[l] = (int32_t)lsp.size();
            lsp.insert(lsp.end(), lanes[l].begin(), lanes[l].end());
        }
        lptr[32] = (int32_t)lsp.size();
    }
    // reaction records, slot-major words
    constexpr size_t kW32 = sizeof(RxnF32) / 4;
    std::vector<uint32_t> rt(kW32 * order.size(), 0);
    for (size_t sl = 0; sl < order.size(); ++sl) {
        if (order[sl] < 0) continue;
        uint32_t w[kW32];
        memcpy(w, &r32[order[sl]], sizeof(RxnF32));
        for (size_t q = 0; q < kW32; ++q) rt[q * order.size() + sl] = w[q];
    }
    constexpr size_t kW64 = sizeof(RxnF64) / 4;
    std::vector<uint32_t> rt64(kW64 * order.size(), 0);
    for (size_t sl = 0; sl < order.size(); ++sl) {
        if (order[sl] < 0) continue;
        uint32_t w[kW64];
        memcpy(w, &r64[order[sl]], sizeof(RxnF64));
        for (size_t q = 0; q < kW64; ++q) rt64[q * order.size() + sl] = w[q];
    }
    size_t o_ord = align(o_w + sizeof(double) * ns);
    size_t o_gptr = align(o_ord + sizeof(int32_t) * order.size());
    size_t o_gslot = align(o_gptr + sizeof(int32_t) * gptr.size());
    size_t o_gnu = align(o_gslot + sizeof(int32_t) * nge);
    size_t o_cptr = align(o_gnu + sizeof(double) * nge);
    size_t o_crxn = align(o_cptr + sizeof(int32_t) * cptr.size());
    size_t o_cnu = align(o_crxn + sizeof(int32_t) * nce);
    size_t o_lptr = align(o_cnu + sizeof(float) * nce);
    size_t o_lsp = align(o_lptr + sizeof(int32_t) * lptr.size());
    size_t o_rt = align(o_lsp + sizeof(int32_t) * (lsp.size() ? lsp.size() : 1));
    size_t o_rt64 = align(o_rt + sizeof(uint32_t) * rt.size());
    size_t o_sdptr = align(o_rt64 + sizeof(uint32_t) * rt64.size());
    size_t o_sdrxn = align(o_sdptr + sizeof(int32_t) * sdptr.size());
    size_t o_sdnuf = align(o_sdrxn + sizeof(int32_t) * nsd);
    size_t o_sdnur = align(o_sdnuf + sizeof(float) * nsd);
    size_t o_tsptr = align(o_sdnur + sizeof(float) * nsd);
    size_t o_tsrxn = align(o_tsptr + sizeof(int32_t) * tsptr.size());
    size_t o_tse = align(o_tsrxn + sizeof(int32_t) * nts);
    size_t total = align(o_tse + sizeof(double) * nts);
    std::vector<unsigned char> h(total, 0);
    memcpy(h.data() + o_r64, r64.data(), sizeof(RxnF64) * nr);
    memcpy(h.data() + o_s32, s32.data(), sizeof(SpecF32) * ns);
    if (!tb_sp.empty()) {
        memcpy(h.data() + o_tbsp, tb_sp.data(), sizeof(uint16_t) * tb_sp.size());
        memcpy(h.data() + o_tbe64, tb_e64.data(), sizeof(double) * tb_e64.size());
        memcpy(h.data() + o_tbe32, tb_e32.data(), sizeof(float) * tb_e32.size());
    }
    memcpy(h.data() + o_invw, invW.data(), sizeof(double) * ns);
    memcpy(h.data() + o_rint, rint.data(), sizeof(RxnInt) * nr);
    memcpy(h.data() + o_nasa, d->nasa7, sizeof(double) * 14 * ns);
    memcpy(h.data() + o_w, d->mol_weight, sizeof(double) * ns);
    memcpy(h.data() + o_ord, order.data(), sizeof(int32_t) * order.size());
    memcpy(h.data() + o_gptr, gptr.data(), sizeof(int32_t) * gptr.size());
    if (!gslot.empty()) {
        memcpy(h.data() + o_gslot, gslot.data(), sizeof(int32_t) * gslot.size());
        memcpy(h.data() + o_gnu, gnu.data(), sizeof(double) * gnu.size());
    }
    memcpy(h.data() + o_cptr, cptr.data(), sizeof(int32_t) * cptr.size());
    memcpy(h.data() + o_lptr, lptr.data(), sizeof(int32_t) * lptr.size());
    if (!lsp.empty()) memcpy(h.data() + o_lsp, lsp.data(), sizeof(int32_t) * lsp.size());
    memcpy(h.data() + o_rt, rt.data(), sizeof(uint32_t) * rt.size());
    memcpy(h.data() + o_rt64, rt64.data(), sizeof(uint32_t) * rt64.size());
    if (!crxn.empty()) {
        memcpy(h.data() + o_crxn, crxn.data(), sizeof(int32_t) * crxn.size());
        memcpy(h.data() + o_cnu, cnu.data(), sizeof(float) * cnu.size());
    }
    memcpy(h.data() + o_sdptr, sdptr.data(), sizeof(int32_t) * sdptr.size());
    memcpy(h.data() + o_tsptr, tsptr.data(), sizeof(int32_t) * tsptr.size());
    if (!sdrxn.empty()) {
        memcpy(h.data() + o_sdrxn, sdrxn.data(), sizeof(int32_t) * sdrxn.size());
        memcpy(h.data() + o_sdnuf, sdnuf.data(), sizeof(float) * sdnuf.size());
        memcpy(h.data() + o_sdnur, sdnur.data(), sizeof(float) * sdnur.size());
    }
    if (!tsrxn.empty()) {
        memcpy(h.data() + o_tsrxn, tsrxn.data(), sizeof(int32_t) * tsrxn.size());
        memcpy(h.data() + o_tse, tse.data(), sizeof(double) * tse.size());
    }

    chem_mech *m = new (std::nothrow) chem_mech();
    if (!m) return set_error(CHEM_ENOMEM, "host allocation failed");
    m->ns = ns;
    m->nr = nr;
    m->t_mid = d->t_mid;
    m->p_ref = d->p_ref;
    m->have_bf16 = false;
    m->bf16_wide = false;
    m->bf16 = nullptr;
    m->vt.ok = false;
    m->d_f32t = nullptr;
    if (cudaGetDevice(&m->device) != cudaSuccess) {
        delete m;
        return set_error(CHEM_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(cudaGetLastError()));
    }
    cudaError_t e = cudaMalloc(&m->d_blob, total);
    if (e != cudaSuccess) {
        delete m;
        return set_error(CHEM_ENOMEM, "cudaMalloc(%zu): %s", total, cudaGetErrorString(e));
    }
    e = cudaMemcpy(m->d_blob, h.data(), total, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(m->d_blob);
        delete m;
        return set_error(CHEM_ECUDA, "cudaMemcpy: %s", cudaGetErrorString(e));
    }
    m->device_bytes = total;
    unsigned char *base = (unsigned char *)m->d_blob;
    m->v64.ns = ns;
    m->v64.nr = nr;
    m->v64.rxn = (const RxnF64 *)(base + o_r64);
    m->v64.tb_sp = (const uint16_t *)(base + o_tbsp);
    m->v64.tb_e = (const double *)(base + o_tbe64);
    m->v64.invW = (const double *)(base + o_invw);
    m->v64.t_mid = d->t_mid;
    m->v32.ns = ns;
    m->v32.nr = nr;
    m->v32.spec = (const SpecF32 *)(base + o_s32);
    m->v32.tb_sp = (const uint16_t *)(base + o_tbsp);
    m->v32.tb_e = (const float *)(base + o_tbe32);
    m->v32.t_mid = (float)d->t_mid;
    m->v32.lg2_pref_R = dsplit(log2(d->p_ref / kR));
    m->v32.col_ptr = (const int32_t *)(base + o_cptr);
    m->v32.col_rxn = (const int32_t *)(base + o_crxn);
    m->v32.col_nu = (const float *)(base + o_cnu);
    m->v32.lane_ptr = (const int32_t *)(base + o_lptr);
    m->v32.lane_sp = (const int32_t *)(base + o_lsp);
    m->v32.rxn_t = (const uint32_t *)(base + o_rt);
    m->v32.n_slots = (int32_t)order.size();
    m->v64.rxn_t = (const uint32_t *)(base + o_rt64);
    m->v64.n_slots = m->v32.n_slots;
    m->v64.col_ptr = m->v32.col_ptr;
    m->v64.col_rxn = m->v32.col_rxn;
    m->v64.col_nu = m->v32.col_nu;
    m->v64.lane_ptr = m->v32.lane_ptr;
    m->v64.lane_sp = m->v32.lane_sp;
    m->v64.sd_ptr = (const int32_t *)(base + o_sdptr);
    m->v64.sd_rxn = (const int32_t *)(base + o_sdrxn);
    m->v64.sd_nuf = (const float *)(base + o_sdnuf);
    m->v64.sd_nur = (const float *)(base + o_sdnur);
    m->v64.ts_ptr = (const int32_t *)(base + o_tsptr);
    m->v64.ts_rxn = (const int32_t *)(base + o_tsrxn);
    m->v64.ts_e = (const double *)(base + o_tse);
    m->vint.rxn = (const RxnInt *)(base + o_rint);
    m->vint.nasa = (const double *)(base + o_nasa);
    m->vint.W = (const double *)(base + o_w);
    m->vint.ok = int_ok;
    m->vint.order = (const int32_t *)(base + o_ord);
    m->vint.n_slots = (int32_t)order.size();
    m->vint.gptr = (const int32_t *)(base + o_gptr);
    m->vint.gent_slot = (const int32_t *)(base + o_gslot);
    m->vint.gent_nu = (const double *)(base + o_gnu);

    st = bf16_build_tables(m, d);
    if (st != CHEM_OK && st != CHEM_EUNSUPPORTED) {
        cudaFree(m->d_blob);
        delete m;
        return st;
    }
    st = f32t_build_tables(m, d);
    if (st != CHEM_OK) {
        bf16_free_tables(m);
        cudaFree(m->d_blob);
        delete m;
        return st;
    }
    clear_error();
    *out = m;
    return CHEM_OK;
}

extern "C" chem_status chem_mechanism_free(chem_mech *m)
{
    clear_error();
    if (!m) return CHEM_OK;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != m->device) cudaSetDevice(m->device);
    cudaDeviceSynchronize();
    bf16_free_tables(m);
    f32t_free_tables(m);
    cudaError_t e = cudaFree(m->d_blob);
    if (cur >= 0 && cur != m->device) cudaSetDevice(cur);
    delete m;
    if (e != cudaSuccess) return set_error(CHEM_ECUDA, "cudaFree: %s", cudaGetErrorString(e));
    return CHEM_OK;
}

extern "C" chem_status chem_mechanism_info(const chem_mech *m, int32_t *ns, int32_t *nr,
                                           size_t *bytes)
{
    clear_error();
    if (!m) return set_error(CHEM_EINVAL, "mechanism is NULL");
    if (ns) *ns = m->ns;
    if (nr) *nr = m->nr;
    if (bytes) *bytes = m->device_bytes;
    return CHEM_OK;
}
