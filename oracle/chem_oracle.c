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
void orc_cell_detail(const orc_mech *m, double T, const double *C, double *g_RT,
                     double *lnkf_out, double *lnKc_out, double *M_out, double *kf_out,
                     double *kr_out, double *qf_out, double *qr_out, double *omega)
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
