// Builds the thread-per-cell FP32 kernel's tables (paper_2008_08483_gb300/csrc/
// chem_f32t_tables.h) for tests/test_f32t_tables.py.  Input (stdin, whitespace separated):
// ns nr t_mid p_ref, then mol_weight[ns], nu_f[nr][ns], nu_r[nr][ns], arrh[nr][3], kind[nr],
// reversible[nr], eff[nr][ns], arrh_low[nr][3], troe[nr][4], nasa7[ns][2][7].  Output: "ok",
// the sizes and constants, then one line per record, species, efficiency entry and falloff
// record (floats printed exactly, %.9g).
#include <stdio.h>

#include <vector>

#include "chem_f32t_tables.h"

template <class T>
static bool read_all(std::vector<T> &v, const char *fmt)
{
    for (auto &x : v)
        if (scanf(fmt, &x) != 1) return false;
    return true;
}

int main()
{
    int ns = 0, nr = 0;
    double t_mid = 0, p_ref = 0;
    if (scanf("%d %d %lf %lf", &ns, &nr, &t_mid, &p_ref) != 4) return 1;
    std::vector<double> W(ns), arrh(3 * nr), eff((size_t)nr * ns), low(3 * nr), troe(4 * nr),
        nasa((size_t)ns * 14);
    std::vector<int> nuf((size_t)nr * ns), nur((size_t)nr * ns), kind(nr), rev(nr);
    if (!read_all(W, "%lf") || !read_all(nuf, "%d") || !read_all(nur, "%d") ||
        !read_all(arrh, "%lf") || !read_all(kind, "%d") || !read_all(rev, "%d") ||
        !read_all(eff, "%lf") || !read_all(low, "%lf") || !read_all(troe, "%lf") ||
        !read_all(nasa, "%lf"))
        return 1;
    chem_mech_desc d;
    memset(&d, 0, sizeof d);
    d.n_species = ns;
    d.n_reactions = nr;
    d.mol_weight = W.data();
    d.nu_f = nuf.data();
    d.nu_r = nur.data();
    d.arrh = arrh.data();
    d.kind = kind.data();
    d.reversible = rev.data();
    d.eff = eff.data();
    d.arrh_low = low.data();
    d.troe = troe.data();
    d.nasa7 = nasa.data();
    d.t_mid = t_mid;
    d.p_ref = p_ref;
    using namespace chem;
    f32t::Tables t;
    if (!f32t::build_tables(&d, t)) {
        printf("ok 0\n");
        return 0;
    }
    const F32TView &v = t.v;
    printf("ok 1\n");
    printf("sizes %d %d %d %d\n", v.n_rec, v.n_tb, v.n_fall, (int)t.sp.size());
    printf("const %.9g %.9g %.9g %.9g %.9g %.9g %.9g %.9g %.9g %.9g %.9g %.9g\n", v.lg2T0.x,
           v.lg2T0.y, v.invT0.x, v.invT0.y, v.lg2R.x, v.lg2R.y, v.lg2_pref_R.x, v.lg2_pref_R.y,
           v.log2e.x, v.log2e.y, v.Tc[0], v.Tc[1]);
    for (size_t i = 0; i < t.rx.size(); ++i) {
        const RxnT &r = t.rx[i];
        printf("rec %d %.9g %.9g %.9g %.9g %.9g %u %u %.9g", t.order[i], r.kf.x, r.kf.y, r.kf.z,
               r.kf.w, r.b, r.meta, r.tb, r.rb);
        for (int e = 0; e < 12; ++e) {
            float nu;
            memcpy(&nu, &r.ent[2 * e + 1], 4);
            printf(" %d %.9g", r.ent[2 * e], nu);
        }
        printf("\n");
    }
    for (const SpecT &s : t.sp) {
        printf("spec");
        for (int rg = 0; rg < 2; ++rg)
            printf(" %.9g %.9g %.9g %.9g %.9g %.9g %.9g %.9g %.9g %.9g %.9g %.9g", s.ga[rg].x,
                   s.ga[rg].y, s.ga[rg].z, s.ga[rg].w, s.gb[rg].x, s.gb[rg].y, s.gb[rg].z,
                   s.gb[rg].w, s.gc[rg].x, s.gc[rg].y, s.gc[rg].z, s.gc[rg].w);
        printf("\n");
    }
    for (const int2 &e : t.tb) {
        float x;
        memcpy(&x, &e.y, 4);
        printf("tb %d %.9g\n", e.x, x);
    }
    for (const FallT &f : t.fall)
        printf("fall %.9g %.9g %.9g %.9g %.9g %.9g %.9g %.9g %.9g %.9g %.9g %.9g\n", f.k0.x, f.k0.y,
               f.k0.z, f.k0.w, f.t0.x, f.t0.y, f.t0.z, f.t0.w, f.t1.x, f.t1.y, f.t1.z, f.t1.w);
    return 0;
}
