/*
 * chem_oracle.c -- FP64 CPU oracle for the batched chemical source term.
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the package smoke check and the
 * benchmark's CPU-baseline / reference leg load this file's library.  It shares
 * no code, header, table or helper with the CUDA library, and neither side
 * includes or links the other.
 *
 * It computes the plain definition of the net production rates, one cell and
 * one reaction at a time, in double precision, with no matrices and no
 * reordering:
 *   - mechanism sum_k nu'_kj S_k <=> sum_k nu''_kj S_k                 (Eq. 1)
 *   - omega_k = sum_j (nu''_kj - nu'_kj) q_net,j                        (Eq. 2)
 *   - q_net,j = k_f,j prod_k C_k^nu'_kj - k_r,j prod_k C_k^nu''_kj      (Eq. 3)
 *   - k_f,j = A_j T^b_j exp(-E_j / (R T))                               (Eq. 5)
 *   - k_r,j = k_f,j / K_c,j                                             (Eq. 7)
 *   - K_c,j = (p_ref / R T)^(sum_k nu_kj) exp(dS_j/R - dH_j/(R T))      (Eq. 8)
 *     with dS/R - dH/(RT) = -sum_k nu_kj g_k/(RT) from NASA-7 thermo (Eq. 10,
 *     two temperature ranges split at T_mid)
 *   - third-body reactions multiply k_f and k_r by M_j = sum_k eff_kj C_k,
 *     falloff reactions use M_j in the reduced pressure (Lindemann or Troe),
 *     irreversible reactions have k_r = 0                              (Sec. 2.4)
 *
 * The paper gives no formula for the Troe function; the oracle uses the
 * Gilbert-Luther-Troe form (F_cent with three exponentials, c = -0.4 - 0.67
 * log10 F_cent, n = 0.75 - 1.27 log10 F_cent, d = 0.14).  Negative mass
 * fractions are clipped to zero before C is formed.
 *
 * Units are cgs: mol, cm^3, s, K, erg.  R = 8.31446261815324e7 erg/(mol K).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_R 8.31446261815324e7

typedef struct {
    int ns, nr;
    const double *W;        /* [ns] molecular weights, g/mol */
    const int32_t *nu_f;    /* [nr][ns] reactant coefficients nu' */
    const int32_t *nu_r;    /* [nr][ns] product coefficients nu'' */
    const double *arrh;     /* [nr][3] ln A, b, E/R */
    const int32_t *kind;    /* [nr] 0 elementary, 1 third body, 2 Lindemann, 3 Troe */
    const int32_t *rev;     /* [nr] 1 reversible */
    const double *eff;      /* [nr][ns] third-body efficiencies */
    const double *arrh_low; /* [nr][3] low-pressure ln A0, b0, E0/R */
    const double *troe;     /* [nr][4] alpha, T***, T*, T** (T** <= 0: absent) */
    const double *nasa;     /* [ns][2][7] NASA-7 sets: [0] T < t_mid, [1] T >= t_mid */
    double t_mid, p_ref;
} orc_mech;

/* NASA-7 polynomials (Eq. 10): per species cp/R, h/(RT), s/R and g/(RT) = h/(RT) - s/R. */
void orc_thermo(const orc_mech *m, double T, double *cp_R, double *h_RT, double *s_R,
                double *g_RT)
{
    for (int k = 0; k < m->ns; ++k) {
        const double *a = m->nasa + (size_t)k * 14 + (T < m->t_mid ? 0 : 7);
        double cp = a[0] + a[1] * T + a[2] * T * T + a[3] * T * T * T + a[4] * T * T * T * T;
        double h = a[0] + a[1] * T / 2.0 + a[2] * T * T / 3.0 + a[3] * T * T * T / 4.0 +
                   a[4] * T * T * T * T / 5.0 + a[5] / T;
        double s = a[0] * log(T) + a[1] * T + a[2] * T * T / 2.0 + a[3] * T * T * T / 3.0 +
                   a[4] * T * T * T * T / 4.0 + a[6];
        if (cp_R) cp_R[k] = cp;
        if (h_RT) h_RT[k] = h;
        if (s_R) s_R[k] = s;
        if (g_RT) g_RT[k] = h - s;
    }
}

/* Concentrations from (T, P, Y): rho = P Wbar / (R T), C_k = rho Y_k / W_k, with
 * Wbar = 1 / sum_k Y_k / W_k.  Negative Y_k count as zero; all-zero Y gives C = 0. */
void orc_concentrations(const orc_mech *m, double T, double P, const double *Y, double *C)
{
    double sum = 0.0;
    for (int k = 0; k < m->ns; ++k) {
        double y = Y[k] > 0.0 ? Y[k] : 0.0;
        sum += y / m->W[k];
    }
    double ctot = P / (ORC_R * T);
    for (int k = 0; k < m->ns; ++k) {
        double y = Y[k] > 0.0 ? Y[k] : 0.0;
        C[k] = sum > 0.0 ? ctot * (y / m->W[k]) / sum : 0.0;
    }
}

/* Troe falloff factor F(T, Pr) in the Gilbert-Luther-Troe form. */
double orc_troe_F(const double *tp, double T, double Pr)
{
    double alpha = tp[0], T3 = tp[1], T1 = tp[2], T2 = tp[3];
    double Fcent = (1.0 - alpha) * exp(-T / T3) + alpha * exp(-T / T1);
    if (T2 > 0.0) Fcent += exp(-T2 / T);
    double lFc = log10(Fcent);
    double c = -0.4 - 0.67 * lFc;
    double n = 0.75 - 1.27 * lFc;
    double x = log10(Pr) + c;
    double f1 = x / (n - 0.14 * x);
    return pow(10.0, lFc / (1.0 + f1 * f1));
}

/*
 * Everything for one cell at (T, C).  Per reaction: ln k_f of the high-pressure /
 * plain Arrhenius expression, ln K_c, the third-body concentration M (1 when the
 * reaction has none), the effective forward and reverse rate constants (with M or
 * the falloff factor applied), q_f and q_r.  Then omega (Eq. 2).  Any output
 * pointer may be NULL.  g_RT is scratch of ns doubles.
 */
static void orc_cell_detail_kc(const orc_mech *m, double T, const double *C, double *g_RT,
                               const double *lnKc_in, double *lnkf_out, double *lnKc_out,
                               double *M_out, double *kf_out, double *kr_out, double *qf_out,
                               double *qr_out, double *omega);

void orc_cell_detail(const orc_mech *m, double T, const double *C, double *g_RT,
                     double *lnkf_out, double *lnKc_out, double *M_out, double *kf_out,
                     double *kr_out, double *qf_out, double *qr_out, double *omega)
{
    orc_cell_detail_kc(m, T, C, g_RT, NULL, lnkf_out, lnKc_out, M_out, kf_out, kr_out, qf_out,
                       qr_out, omega);
}

/* As orc_cell_detail, with ln K_c of every reaction given (lnKc_in, e.g. from the
 * approximate network of Sec. 2.3) instead of computed from the thermo (Eq. 8). */
static void orc_cell_detail_kc(const orc_mech *m, double T, const double *C, double *g_RT,
                               const double *lnKc_in, double *lnkf_out, double *lnKc_out,
                               double *M_out, double *kf_out, double *kr_out, double *qf_out,
                               double *qr_out, double *omega)
{
    const int ns = m->ns;
    orc_thermo(m, T, NULL, NULL, NULL, g_RT);
    double ln_pref_RT = log(m->p_ref / (ORC_R * T));
    if (omega)
        for (int k = 0; k < ns; ++k) omega[k] = 0.0;
    for (int j = 0; j < m->nr; ++j) {
        const int32_t *nf = m->nu_f + (size_t)j * ns;
        const int32_t *nr = m->nu_r + (size_t)j * ns;
        const double *ar = m->arrh + (size_t)j * 3;
        /* Eq. 5 */
        double kinf = exp(ar[0]) * pow(T, ar[1]) * exp(-ar[2] / T);
        double M = 1.0, kf = kinf;
        int kind = m->kind[j];
        if (kind != 0) {
            M = 0.0;
            for (int k = 0; k < ns; ++k) M += m->eff[(size_t)j * ns + k] * C[k];
        }
        if (kind == 1) {
            kf = kinf * M;
        } else if (kind == 2 || kind == 3) {
            const double *al = m->arrh_low + (size_t)j * 3;
            double k0 = exp(al[0]) * pow(T, al[1]) * exp(-al[2] / T);
            double Pr = k0 * M / kinf;
            if (Pr > 0.0) {
                double F = (kind == 3) ? orc_troe_F(m->troe + (size_t)j * 4, T, Pr) : 1.0;
                kf = kinf * (Pr / (1.0 + Pr)) * F;
            } else {
                kf = 0.0;
            }
        }
        /* Eq. 8: ln K_c = -sum_k nu_kj g_k/RT + (sum_k nu_kj) ln(p_ref / RT) */
        double lnKc = 0.0;
        int dnu = 0;
        for (int k = 0; k < ns; ++k) {
            int nu = nr[k] - nf[k];
            if (nu) {
                lnKc -= nu * g_RT[k];
                dnu += nu;
            }
        }
        lnKc += dnu * ln_pref_RT;
        if (lnKc_in) lnKc = lnKc_in[j];
        /* Eq. 7 and the irreversibility indicator of Sec. 2.4 */
        double kr = m->rev[j] ? kf / exp(lnKc) : 0.0;
        /* Eq. 3 */
        double qf = kf, qr = kr;
        for (int k = 0; k < ns; ++k) {
            if (nf[k]) qf *= pow(C[k], (double)nf[k]);
            if (nr[k]) qr *= pow(C[k], (double)nr[k]);
        }
        if (lnkf_out) lnkf_out[j] = log(kinf);
        if (lnKc_out) lnKc_out[j] = lnKc;
        if (M_out) M_out[j] = M;
        if (kf_out) kf_out[j] = kf;
        if (kr_out) kr_out[j] = kr;
        if (qf_out) qf_out[j] = qf;
        if (qr_out) qr_out[j] = qr;
        /* Eq. 2 */
        if (omega) {
            double qnet = qf - qr;
            for (int k = 0; k < ns; ++k) {
                int nu = nr[k] - nf[k];
                if (nu) omega[k] += nu * qnet;
            }
        }
    }
}

/* ---- batched drivers (threads over contiguous cell ranges) ---------------- */

typedef struct {
    const orc_mech *m;
    int64_t lo, hi;
    const double *T, *P, *Y;   /* Y holds C when P == NULL */
    int64_t ldY;
    double *omega;
    int64_t ldO;
} orc_job;

static void *orc_worker(void *arg)
{
    orc_job *jb = (orc_job *)arg;
    const orc_mech *m = jb->m;
    double *C = (double *)malloc(sizeof(double) * (size_t)m->ns * 2);
    if (!C) return (void *)1;
    double *g = C + m->ns;
    for (int64_t i = jb->lo; i < jb->hi; ++i) {
        const double *row = jb->Y + i * jb->ldY;
        if (jb->P) {
            orc_concentrations(m, jb->T[i], jb->P[i], row, C);
        } else {
            for (int k = 0; k < m->ns; ++k) C[k] = row[k];
        }
        orc_cell_detail(m, jb->T[i], C, g, NULL, NULL, NULL, NULL, NULL, NULL, NULL,
                        jb->omega + i * jb->ldO);
    }
    free(C);
    return NULL;
}

static int orc_run(const orc_mech *m, int64_t n, const double *T, const double *P,
                   const double *Y, int64_t ldY, double *omega, int64_t ldO, int nthreads)
{
    if (n <= 0) return 0;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 1024) nthreads = 1024;
    if ((int64_t)nthreads > n) nthreads = (int)n;
    pthread_t th[1024];
    orc_job jobs[1024];
    int rc = 0;
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].m = m;
        jobs[t].lo = n * t / nthreads;
        jobs[t].hi = n * (t + 1) / nthreads;
        jobs[t].T = T;
        jobs[t].P = P;
        jobs[t].Y = Y;
        jobs[t].ldY = ldY;
        jobs[t].omega = omega;
        jobs[t].ldO = ldO;
    }
    for (int t = 1; t < nthreads; ++t)
        if (pthread_create(&th[t], NULL, orc_worker, &jobs[t]) != 0) return -1;
    if (orc_worker(&jobs[0]) != NULL) rc = -1;
    for (int t = 1; t < nthreads; ++t) {
        void *r = NULL;
        pthread_join(th[t], &r);
        if (r) rc = -1;
    }
    return rc;
}

/* omega [n][ldO] from cell states T [n] (K), P [n] (dyn/cm^2), Y [n][ldY]. */
int orc_source_term_tpy(const orc_mech *m, int64_t n, const double *T, const double *P,
                        const double *Y, int64_t ldY, double *omega, int64_t ldO, int nthreads)
{
    return orc_run(m, n, T, P, Y, ldY, omega, ldO, nthreads);
}

/* omega [n][ldO] from T [n] and concentrations C [n][ldC] (mol/cm^3). */
int orc_source_term_tc(const orc_mech *m, int64_t n, const double *T, const double *C,
                       int64_t ldC, double *omega, int64_t ldO, int nthreads)
{
    return orc_run(m, n, T, NULL, C, ldC, omega, ldO, nthreads);
}

/* ---- analytic Jacobian of omega with respect to (ln C, T) --------------------------------
 *
 * For each reaction, with q_f = k_f prod C^nu' and q_r = k_f / K_c prod C^nu'':
 *   d ln q_f / d ln C_m = nu'_m + d ln k_f / d ln C_m,   d ln q_r / d ln C_m = nu''_m + same
 *   d ln q_f / dT = d ln k_f / dT,                       d ln q_r / dT = d ln k_f / dT - d ln K_c / dT
 * with d ln k_inf / dT = b/T + (E/R)/T^2 (Eq. 5), d ln K_c / dT = sum_k nu_k h_k/(R T^2) - dnu/T
 * (Eq. 8, since d(g/RT)/dT = -h/(R T^2)), d ln M / d ln C_m = eff_m C_m / M for third-body
 * reactions, and for falloff reactions the chain rule through Pr = k0 M / k_inf and the
 * Troe function.  Then d omega_k = sum_j nu_kj (d q_f - d q_r) (Eq. 2).
 * dw_dlnC is [ns][ns] (row: species of omega, column: ln C_m), dw_dT is [ns].
 */

/* d log10 F / d log10 Pr and d log10 F / dT (at fixed Pr) of the Troe function */
static void orc_troe_dF(const double *tp, double T, double Pr, double *dlF_dlPr, double *dlF_dT)
{
    double alpha = tp[0], T3 = tp[1], T1 = tp[2], T2 = tp[3];
    double e3 = exp(-T / T3), e1 = exp(-T / T1);
    double Fc = (1.0 - alpha) * e3 + alpha * e1;
    double dFc = -(1.0 - alpha) / T3 * e3 - alpha / T1 * e1;
    if (T2 > 0.0) {
        double e2 = exp(-T2 / T);
        Fc += e2;
        dFc += T2 / (T * T) * e2;
    }
    double L = log10(Fc);
    double dL_dT = dFc / (Fc * log(10.0));
    double c = -0.4 - 0.67 * L, n = 0.75 - 1.27 * L;
    double x = log10(Pr) + c;
    double D = n - 0.14 * x;
    double f1 = x / D;
    double g = 1.0 + f1 * f1;
    /* df1/dx at fixed L: (D + 0.14 x) / D^2 = n / D^2 */
    double df1_dx = n / (D * D);
    *dlF_dlPr = -L * 2.0 * f1 / (g * g) * df1_dx;
    /* through L: dx/dL = -0.67, dD/dL = -1.27 + 0.14 * 0.67 */
    double dD_dL = -1.27 + 0.14 * 0.67;
    double df1_dL = (-0.67 * D - x * dD_dL) / (D * D);
    double dlF_dL = 1.0 / g - L * 2.0 * f1 / (g * g) * df1_dL;
    *dlF_dT = dlF_dL * dL_dT;
}

void orc_jacobian_tc(const orc_mech *m, double T, const double *C, double *h_RT,
                     double *g_RT, double *dw_dlnC, double *dw_dT)
{
    const int ns = m->ns;
    orc_thermo(m, T, NULL, h_RT, NULL, g_RT);
    double ln_pref_RT = log(m->p_ref / (ORC_R * T));
    for (int i = 0; i < ns * ns; ++i) dw_dlnC[i] = 0.0;
    for (int k = 0; k < ns; ++k) dw_dT[k] = 0.0;
    double *dmod = (double *)malloc(sizeof(double) * (size_t)ns);   /* d ln(modifier)/d ln C */
    if (!dmod) return;
    for (int j = 0; j < m->nr; ++j) {
        const int32_t *nf = m->nu_f + (size_t)j * ns;
        const int32_t *nr = m->nu_r + (size_t)j * ns;
        const double *ar = m->arrh + (size_t)j * 3;
        double kinf = exp(ar[0]) * pow(T, ar[1]) * exp(-ar[2] / T);
        double dlkinf_dT = ar[1] / T + ar[2] / (T * T);
        double kf = kinf, dlkf_dT = dlkinf_dT;
        int kind = m->kind[j];
        for (int k = 0; k < ns; ++k) dmod[k] = 0.0;
        if (kind != 0) {
            double M = 0.0;
            for (int k = 0; k < ns; ++k) M += m->eff[(size_t)j * ns + k] * C[k];
            if (kind == 1) {
                kf = kinf * M;
                for (int k = 0; k < ns; ++k)
                    dmod[k] = M > 0.0 ? m->eff[(size_t)j * ns + k] * C[k] / M : 0.0;
            } else {
                const double *al = m->arrh_low + (size_t)j * 3;
                double k0 = exp(al[0]) * pow(T, al[1]) * exp(-al[2] / T);
                double Pr = k0 * M / kinf;
                if (!(Pr > 0.0)) continue;              /* k_f = 0: no contribution */
                double F = 1.0, dlF_dlPr = 0.0, dlF_dT = 0.0;   /* log10 F derivatives */
                if (kind == 3) {
                    F = orc_troe_F(m->troe + (size_t)j * 4, T, Pr);
                    orc_troe_dF(m->troe + (size_t)j * 4, T, Pr, &dlF_dlPr, &dlF_dT);
                }
                kf = kinf * (Pr / (1.0 + Pr)) * F;
                double dmod_dlPr = 1.0 / (1.0 + Pr) + dlF_dlPr;
                double dlPr_dT = (al[1] - ar[1]) / T + (al[2] - ar[2]) / (T * T);
                dlkf_dT = dlkinf_dT + dmod_dlPr * dlPr_dT + dlF_dT * log(10.0);
                for (int k = 0; k < ns; ++k)
                    dmod[k] = dmod_dlPr * m->eff[(size_t)j * ns + k] * C[k] / M;
            }
        }
        double lnKc = 0.0, dlKc_dT = 0.0;
        int dnu = 0;
        for (int k = 0; k < ns; ++k) {
            int nu = nr[k] - nf[k];
            if (nu) {
                lnKc -= nu * g_RT[k];
                dlKc_dT += nu * h_RT[k] / T;
                dnu += nu;
            }
        }
        lnKc += dnu * ln_pref_RT;
        dlKc_dT -= dnu / T;
        double kr = m->rev[j] ? kf / exp(lnKc) : 0.0;
        double qf = kf, qr = kr;
        for (int k = 0; k < ns; ++k) {
            if (nf[k]) qf *= pow(C[k], (double)nf[k]);
            if (nr[k]) qr *= pow(C[k], (double)nr[k]);
        }
        double dqnet_dT = qf * dlkf_dT - qr * (dlkf_dT - dlKc_dT);
        for (int k = 0; k < ns; ++k) {
            int nu = nr[k] - nf[k];
            if (!nu) continue;
            dw_dT[k] += nu * dqnet_dT;
            double *row = dw_dlnC + (size_t)k * ns;
            for (int mm = 0; mm < ns; ++mm) {
                double d = qf * (nf[mm] + dmod[mm]) - qr * (nr[mm] + dmod[mm]);
                row[mm] += nu * d;
            }
        }
    }
    free(dmod);
}

/* ---- constant-pressure adiabatic 0-D reactor ---------------------------------------------
 *
 * State y = (T, Y_1 .. Y_ns) at fixed pressure P.  With S = sum_k Y_k / W_k,
 * rho = P / (R T S) and C_k = rho Y_k / W_k:
 *   dY_k / dt = W_k omega_k / rho
 *   dT / dt   = -sum_k H_k omega_k / (rho c_p)
 * with the molar enthalpies H_k = R T (h/RT)_k and the mass heat capacity
 * c_p = sum_k Y_k R (cp/R)_k / W_k.  These keep the mixture enthalpy sum_k Y_k H_k / W_k
 * constant (adiabatic, constant pressure) and sum_k Y_k constant.  The mass-action products
 * take C as it comes, without clipping: the right-hand side is then a polynomial in C and a
 * smooth function of y, as an implicit integrator that may step through small negative mass
 * fractions needs.
 */

/* d/dC_m of prod_k C_k^nu_k, i.e. nu_m C_m^(nu_m - 1) prod_{k != m} C_k^nu_k */
static double orc_dprod(const int32_t *nu, const double *C, int ns, int mcol)
{
    if (!nu[mcol]) return 0.0;
    double p = nu[mcol] * pow(C[mcol], (double)(nu[mcol] - 1));
    for (int k = 0; k < ns; ++k)
        if (k != mcol && nu[k]) p *= pow(C[k], (double)nu[k]);
    return p;
}

/*
 * d omega / dC [ns][ns] and d omega / dT at fixed C [ns], with the mass-action products
 * differentiated directly (no division by C, so C_m = 0 is fine):
 *   d q_f / dC_m = k_f d(prod C^nu')/dC_m + eff_m (d k_f / dM) prod C^nu'
 *   d q_r / dC_m = k_r d(prod C^nu'')/dC_m + eff_m (d k_f / dM) / K_c prod C^nu''
 * with d k_f / dM = k_inf for third-body reactions and k_f (1/(1+Pr) + d log F / d log Pr) / M
 * for falloff reactions; the temperature derivatives are those of orc_jacobian_tc.
 */
void orc_dwdC(const orc_mech *m, double T, const double *C, double *dwdC, double *dwdT)
{
    const int ns = m->ns;
    double *h_RT = (double *)malloc(sizeof(double) * (size_t)ns * 2);
    if (!h_RT) return;
    double *g_RT = h_RT + ns;
    orc_thermo(m, T, NULL, h_RT, NULL, g_RT);
    double ln_pref_RT = log(m->p_ref / (ORC_R * T));
    for (int i = 0; i < ns * ns; ++i) dwdC[i] = 0.0;
    for (int k = 0; k < ns; ++k) dwdT[k] = 0.0;
    for (int j = 0; j < m->nr; ++j) {
        const int32_t *nf = m->nu_f + (size_t)j * ns;
        const int32_t *nr = m->nu_r + (size_t)j * ns;
        const double *ar = m->arrh + (size_t)j * 3;
        const double *eff = m->eff + (size_t)j * ns;
        double kinf = exp(ar[0]) * pow(T, ar[1]) * exp(-ar[2] / T);
        double dlkf_dT = ar[1] / T + ar[2] / (T * T);
        double kf = kinf, dkf_dM = 0.0;
        int kind = m->kind[j];
        if (kind != 0) {
            double M = 0.0;
            for (int k = 0; k < ns; ++k) M += eff[k] * C[k];
            if (kind == 1) {
                kf = kinf * M;
                dkf_dM = kinf;
            } else {
                const double *al = m->arrh_low + (size_t)j * 3;
                double k0 = exp(al[0]) * pow(T, al[1]) * exp(-al[2] / T);
                double Pr = k0 * M / kinf;
                if (!(Pr > 0.0)) continue;
                double F = 1.0, dlF_dlPr = 0.0, dlF_dT = 0.0;
                if (kind == 3) {
                    F = orc_troe_F(m->troe + (size_t)j * 4, T, Pr);
                    orc_troe_dF(m->troe + (size_t)j * 4, T, Pr, &dlF_dlPr, &dlF_dT);
                }
                kf = kinf * (Pr / (1.0 + Pr)) * F;
                double dmod_dlPr = 1.0 / (1.0 + Pr) + dlF_dlPr;
                dkf_dM = kf * dmod_dlPr / M;
                double dlPr_dT = (al[1] - ar[1]) / T + (al[2] - ar[2]) / (T * T);
                dlkf_dT += dmod_dlPr * dlPr_dT + dlF_dT * log(10.0);
            }
        }
        double lnKc = 0.0, dlKc_dT = 0.0;
        int dnu = 0;
        for (int k = 0; k < ns; ++k) {
            int nu = nr[k] - nf[k];
            if (nu) {
                lnKc -= nu * g_RT[k];
                dlKc_dT += nu * h_RT[k] / T;
                dnu += nu;
            }
        }
        lnKc += dnu * ln_pref_RT;
        dlKc_dT -= dnu / T;
        double Kc = exp(lnKc);
        int rev = m->rev[j];
        double kr = rev ? kf / Kc : 0.0;
        double pf = 1.0, pr = 1.0;
        for (int k = 0; k < ns; ++k) {
            if (nf[k]) pf *= pow(C[k], (double)nf[k]);
            if (nr[k]) pr *= pow(C[k], (double)nr[k]);
        }
        double qf = kf * pf, qr = kr * pr;
        double dqnet_dT = qf * dlkf_dT - qr * (dlkf_dT - dlKc_dT);
        double dqnet_dM = dkf_dM * (pf - (rev ? pr / Kc : 0.0));
        for (int k = 0; k < ns; ++k) {
            int nu = nr[k] - nf[k];
            if (!nu) continue;
            dwdT[k] += nu * dqnet_dT;
            double *row = dwdC + (size_t)k * ns;
            for (int mm = 0; mm < ns; ++mm) {
                double d = kf * orc_dprod(nf, C, ns, mm) - kr * orc_dprod(nr, C, ns, mm);
                if (kind != 0) d += eff[mm] * dqnet_dM;
                row[mm] += nu * d;
            }
        }
    }
    free(h_RT);
}

/* Right-hand side f [ns + 1] of the reactor at state y [ns + 1] and pressure P. */
void orc_ode_rhs(const orc_mech *m, double P, const double *y, double *f)
{
    const int ns = m->ns;
    double *buf = (double *)malloc(sizeof(double) * (size_t)ns * 5);
    if (!buf) return;
    double *C = buf, *g = buf + ns, *h_RT = buf + 2 * ns, *cp_R = buf + 3 * ns, *w = buf + 4 * ns;
    const double T = y[0];
    const double *Y = y + 1;
    double S = 0.0;
    for (int k = 0; k < ns; ++k) S += Y[k] / m->W[k];
    double rho = P / (ORC_R * T * S);
    for (int k = 0; k < ns; ++k) C[k] = rho * Y[k] / m->W[k];
    orc_cell_detail(m, T, C, g, NULL, NULL, NULL, NULL, NULL, NULL, NULL, w);
    orc_thermo(m, T, cp_R, h_RT, NULL, NULL);
    double cp = 0.0, Q = 0.0;
    for (int k = 0; k < ns; ++k) {
        cp += Y[k] * ORC_R * cp_R[k] / m->W[k];
        Q += ORC_R * T * h_RT[k] * w[k];
    }
    f[0] = -Q / (rho * cp);
    for (int k = 0; k < ns; ++k) f[1 + k] = m->W[k] * w[k] / rho;
    free(buf);
}

/*
 * Jacobian J [(ns + 1)][(ns + 1)] (row: component of f, column: component of y) of
 * orc_ode_rhs, by the chain rule through C(T, Y) = rho Y / W:
 *   dC_m/dT = -C_m / T,   dC_m/dY_n = rho delta_mn / W_m - C_m / (S W_n)
 *   d(1/rho)/dT = 1/(rho T),   d(1/rho)/dY_n = 1/(rho S W_n)
 *   dH_k/dT = R (cp/R)_k,   d(cp/R)_k/dT = a2 + 2 a3 T + 3 a4 T^2 + 4 a5 T^3
 */
void orc_ode_jac(const orc_mech *m, double P, const double *y, double *J)
{
    const int ns = m->ns, n = ns + 1;
    double *buf = (double *)malloc(sizeof(double) * ((size_t)ns * 10 + (size_t)ns * ns));
    if (!buf) return;
    double *C = buf, *g = buf + ns, *h_RT = buf + 2 * ns, *cp_R = buf + 3 * ns, *w = buf + 4 * ns;
    double *dwdT = buf + 5 * ns, *wT = buf + 6 * ns, *dcp = buf + 7 * ns, *wC = buf + 8 * ns;
    double *dwdC = buf + 10 * ns;
    const double T = y[0];
    const double *Y = y + 1;
    double S = 0.0;
    for (int k = 0; k < ns; ++k) S += Y[k] / m->W[k];
    double rho = P / (ORC_R * T * S);
    for (int k = 0; k < ns; ++k) C[k] = rho * Y[k] / m->W[k];
    orc_cell_detail(m, T, C, g, NULL, NULL, NULL, NULL, NULL, NULL, NULL, w);
    orc_thermo(m, T, cp_R, h_RT, NULL, NULL);
    orc_dwdC(m, T, C, dwdC, dwdT);
    for (int k = 0; k < ns; ++k) {
        const double *a = m->nasa + (size_t)k * 14 + (T < m->t_mid ? 0 : 7);
        dcp[k] = ORC_R * (a[1] + 2.0 * a[2] * T + 3.0 * a[3] * T * T + 4.0 * a[4] * T * T * T);
    }
    /* total derivatives of omega: wT[k] = d omega_k/dT, wC[k] = sum_m dwdC[k][m] C_m */
    for (int k = 0; k < ns; ++k) {
        double s = 0.0;
        for (int mm = 0; mm < ns; ++mm) s += dwdC[(size_t)k * ns + mm] * C[mm];
        wC[k] = s;
        wT[k] = dwdT[k] - s / T;
    }
    double cp = 0.0, Q = 0.0, dcpT = 0.0;
    for (int k = 0; k < ns; ++k) {
        cp += Y[k] * ORC_R * cp_R[k] / m->W[k];
        Q += ORC_R * T * h_RT[k] * w[k];
        dcpT += Y[k] * dcp[k] / m->W[k];
    }
    double rc = rho * cp;
    /* column T */
    {
        double dQ = 0.0;
        for (int k = 0; k < ns; ++k) dQ += ORC_R * cp_R[k] * w[k] + ORC_R * T * h_RT[k] * wT[k];
        double drc = -rc / T + rho * dcpT;
        J[0] = -dQ / rc + Q * drc / (rc * rc);
        for (int k = 0; k < ns; ++k)
            J[(size_t)(1 + k) * n] = m->W[k] * wT[k] / rho + m->W[k] * w[k] / (rho * T);
    }
    /* columns Y_n */
    for (int nn = 0; nn < ns; ++nn) {
        double dQ = 0.0;
        for (int k = 0; k < ns; ++k) {
            double dw = dwdC[(size_t)k * ns + nn] * rho / m->W[nn] - wC[k] / (S * m->W[nn]);
            dQ += ORC_R * T * h_RT[k] * dw;
            J[(size_t)(1 + k) * n + 1 + nn] =
                m->W[k] * dw / rho + m->W[k] * w[k] / (rho * S * m->W[nn]);
        }
        double drc = -rc / (S * m->W[nn]) + rho * ORC_R * cp_R[nn] / m->W[nn];
        J[1 + nn] = -dQ / rc + Q * drc / (rc * rc);
    }
    free(buf);
}

/* omega [n][ldO] from (T, P, Y) with ln K_c given per cell and reaction, lnKc [n][ldK]
 * (one thread; for checks of the approximate-network path). */
int orc_source_term_tpy_kc(const orc_mech *m, int64_t n, const double *T, const double *P,
                           const double *Y, int64_t ldY, const double *lnKc, int64_t ldK,
                           double *omega, int64_t ldO)
{
    double *C = (double *)malloc(sizeof(double) * (size_t)m->ns * 2);
    if (!C) return -1;
    double *g = C + m->ns;
    for (int64_t i = 0; i < n; ++i) {
        orc_concentrations(m, T[i], P[i], Y + i * ldY, C);
        orc_cell_detail_kc(m, T[i], C, g, lnKc + i * ldK, NULL, NULL, NULL, NULL, NULL, NULL,
                           NULL, omega + i * ldO);
    }
    free(C);
    return 0;
}
