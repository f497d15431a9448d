/*
 * chem.h -- C ABI of the GB300 batched chemical source-term library.
 *
 * The library evaluates the net species production rates of a batch of
 * reacting cells, with the cell count as the leading dimension, as in
 * "A Neural Network Inspired Formulation of Chemical Kinetics" (Barwey & Raman):
 *
 *   omega_ik = sum_j nu_kj q_net,ij                                  (Eq. 2)
 *   q_net,ij = exp(sum_k nu'_kj ln C_ik + ln k_f,ij)
 *            - exp(sum_k nu''_kj ln C_ik + ln k_r,ij)                (Eqs. 3-4)
 *   ln k_f,ij = ln A_j + b_j ln T_i - (E_j/R) / T_i                  (Eqs. 5-6)
 *   ln k_r,ij = ln k_f,ij - ln K_c,ij                                (Eq. 7)
 *   ln K_c,ij = -sum_k nu_kj g_k(T_i)/(R T_i)
 *             + (sum_k nu_kj) ln(p_ref / (R T_i))                    (Eqs. 8-11)
 *   g_k/(R T) from two-range NASA-7 polynomials                      (Eq. 10)
 *   third-body concentration M_ij = sum_k eff_kj C_ik multiplies k_f and k_r;
 *   falloff reactions (Lindemann, Troe) use M in the reduced pressure;
 *   irreversible reactions have k_r = 0                              (Sec. 2.4)
 *
 * Units are cgs throughout: mol, cm^3, s, K, erg, dyn/cm^2.
 * R = 8.31446261815324e7 erg/(mol K).  omega is in mol/(cm^3 s).
 *
 * Conventions shared by every entry point:
 *  - Array arguments of the compute calls are DEVICE pointers owned by the
 *    caller, unless the function name ends in _host.  The library never frees
 *    caller memory.
 *  - Row-major, cell-major layouts: Y[i * ldY + k] is species k of cell i.
 *    Leading dimensions count elements and must be >= n_species.
 *  - Element type follows the precision: CHEM_FP64 -> double,
 *    CHEM_FP32 and CHEM_SPLIT_BF16 -> float.
 *  - Work is enqueued on the given CUDA stream (cudaStream_t passed as void*;
 *    NULL is the legacy default stream) and runs asynchronously; argument
 *    errors are reported synchronously before anything is enqueued.
 *  - Every call returns a chem_status; on failure chem_last_error() gives a
 *    message for the calling thread.
 *  - Negative mass fractions count as zero.  A cell whose mass fractions are
 *    all zero has all concentrations zero.
 */
#ifndef CHEM_H
#define CHEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CHEM_ABI_VERSION 1

typedef enum {
    CHEM_OK = 0,
    CHEM_EINVAL = 1,        /* invalid argument or descriptor */
    CHEM_ENOMEM = 2,        /* device or host allocation failed */
    CHEM_ECUDA = 3,         /* CUDA launch or runtime error (text in chem_last_error) */
    CHEM_EUNSUPPORTED = 4,  /* valid request outside what this build supports */
    CHEM_EBUSY = 5,
    CHEM_ETIMEOUT = 6,
    CHEM_ENOTREADY = 7,
    CHEM_ENONCONV = 8
} chem_status;

typedef enum {
    CHEM_FP64 = 0,          /* double I/O and arithmetic (SIMT) */
    CHEM_FP32 = 1,          /* float I/O; SIMT float arithmetic, exponents assembled
                               without rounding their large terms (exact 2^-12-grid heads
                               plus remainders up to 192 species, double-float above) */
    CHEM_SPLIT_BF16 = 2     /* float I/O; the stoichiometric contractions on tcgen05
                               tensor cores with split 16-bit operands and FP32
                               accumulation in tensor memory: log2 X and the Arrhenius /
                               Gibbs features as two FP16 terms, q_net as two BF16 terms */
} chem_precision;

/* Reaction kinds (chem_mech_desc.kind). */
enum { CHEM_RXN_ELEMENTARY = 0, CHEM_RXN_THIRD_BODY = 1, CHEM_RXN_LINDEMANN = 2,
       CHEM_RXN_TROE = 3 };

/*
 * Mechanism descriptor (Eq. 1 and Sec. 2.4).  All pointers are HOST pointers
 * read during chem_mechanism_load only; the library copies what it needs.
 */
typedef struct {
    int32_t n_species;        /* N_S >= 1 */
    int32_t n_reactions;      /* N_R >= 1 */
    int32_t n_elements;       /* >= 0; 0 skips the element-balance check */
    const int32_t *elem_comp; /* [n_species][n_elements] atom counts, or NULL */
    const double *mol_weight; /* [n_species] g/mol, > 0 */
    const int32_t *nu_f;      /* [n_reactions][n_species] reactant coefficients nu' >= 0 */
    const int32_t *nu_r;      /* [n_reactions][n_species] product coefficients nu'' >= 0 */
    const double *arrh;       /* [n_reactions][3] ln A (cgs), b, E/R (K); for falloff
                                 reactions the high-pressure limit */
    const int32_t *kind;      /* [n_reactions] CHEM_RXN_* */
    const int32_t *reversible;/* [n_reactions] 1 reversible, 0 irreversible */
    const double *eff;        /* [n_reactions][n_species] third-body efficiencies, or
                                 NULL for all 1; read for kinds 1-3 only */
    const double *arrh_low;   /* [n_reactions][3] low-pressure ln A0, b0, E0/R for kinds
                                 2-3 (may be NULL when there are none) */
    const double *troe;       /* [n_reactions][4] alpha, T***, T*, T** for kind 3;
                                 T*** > 0 and T* > 0; T** <= 0 means the term is absent */
    const double *nasa7;      /* [n_species][2][7] NASA-7 a1..a7: set 0 for T < t_mid,
                                 set 1 for T >= t_mid */
    double t_mid;             /* K, > 0 */
    double p_ref;             /* standard pressure of the thermo data, dyn/cm^2 (1 bar =
                                 1e6 in the paper, Eq. 8) */
} chem_mech_desc;

typedef struct chem_mech chem_mech;   /* opaque; immutable after load */

/* ABI version of the loaded library (CHEM_ABI_VERSION). */
int32_t chem_abi_version(void);

/*
 * Validate a descriptor and build the device-resident tables on the current
 * CUDA device.  Checks: sizes, coefficient ranges (0..127, at most 8 species
 * with nonzero coefficient per side, at least one reactant), element balance
 * when elem_comp is given, positive weights, Troe temperatures, t_mid, p_ref.
 * The FP64 tables fold the Gibbs layer through the net stoichiometry in double
 * precision (Eqs. 9-11).  On success *out owns host and device memory until
 * chem_mechanism_free.  Errors: CHEM_EINVAL (bad descriptor, message names the
 * reaction), CHEM_ENOMEM, CHEM_ECUDA.  Synchronous.
 */
chem_status chem_mechanism_load(const chem_mech_desc *desc, chem_mech **out);

/* Release a mechanism (NULL is accepted).  Synchronises the device first. */
chem_status chem_mechanism_free(chem_mech *mech);

/* Sizes of a loaded mechanism; any output pointer may be NULL. */
chem_status chem_mechanism_info(const chem_mech *mech, int32_t *n_species,
                                int32_t *n_reactions, size_t *device_bytes);

/*
 * Net production rates omega[n_cells][ldO] from cell states: T[n_cells] (K),
 * P[n_cells] (dyn/cm^2), Y[n_cells][ldY] mass fractions (Eqs. 2-11, Sec. 2.4).
 * Concentrations: C_k = rho Y_k / W_k with rho = P Wbar / (R T).
 * Device pointers; element type double for CHEM_FP64, float otherwise.  Columns
 * n_species..ldO-1 of omega are not written.  n_cells == 0 is a no-op.
 * Errors: CHEM_EINVAL (NULL pointers with n_cells > 0, n_cells < 0,
 * ldY/ldO < n_species, mechanism loaded on another device), CHEM_EUNSUPPORTED
 * (precision not built for this mechanism size: CHEM_FP64 needs 2 n_species + n_reactions
 * <= 3440; CHEM_FP32 takes up to 192 species with at most three species a side and any
 * reaction count (thread-per-cell kernel; its staged species, third-body and falloff tables
 * must fit in shared memory), else needs 5 n_species + n_reactions <= 6752;
 * CHEM_SPLIT_BF16 takes up to 192 species (tables resident in shared memory up to 53,
 * streamed from L2 beyond), with the third-body / falloff reactions within the multiplier
 * slots (8 per 16-reaction share, at most 4 of them falloff) and its shared-memory operands
 * within 227 KB), CHEM_ECUDA (launch failure).
 * Asynchronous on `stream`.
 */
chem_status chem_source_term(const chem_mech *mech, int64_t n_cells, const void *T,
                             const void *P, const void *Y, int64_t ldY, void *omega,
                             int64_t ldO, chem_precision precision, void *stream);

/*
 * Device workspace (bytes) that chem_source_term_host needs for a given chunk size:
 * three stages of T, P, Y and omega rows of chunk_cells cells each.
 */
size_t chem_source_term_host_workspace(const chem_mech *mech, int64_t chunk_cells,
                                       int64_t ldY, chem_precision precision);

/*
 * chem_source_term with HOST arrays (same layouts and element types): the cells are
 * processed in chunks of chunk_cells; each chunk is copied host->device, evaluated and
 * copied back, with the copies of one chunk overlapping the kernel of the next on three
 * library-owned streams.  Host arrays should be page-locked for the copies to overlap.
 * `workspace` is caller-owned device memory of at least
 * chem_source_term_host_workspace(mech, chunk_cells, ldY, precision) bytes, 256-byte
 * aligned; the library allocates nothing per call.  The work is ordered after prior work
 * on `stream`, and `stream` waits for all of it, so synchronising `stream` makes omega
 * valid on the host.  Errors: as chem_source_term, plus CHEM_EINVAL for a NULL or
 * undersized workspace or chunk_cells < 1.
 */
chem_status chem_source_term_host(const chem_mech *mech, int64_t n_cells, const void *T,
                                  const void *P, const void *Y, int64_t ldY, void *omega,
                                  int64_t ldO, chem_precision precision, int64_t chunk_cells,
                                  void *workspace, size_t workspace_bytes, void *stream);

/*
 * Derivatives of omega with respect to the state (T, ln C), where C are the molar
 * concentrations (mol/cm^3, C = exp(ln C)); M = sum_k eff_k C_k for third-body and
 * falloff reactions, so the state fixes omega without P.  Chain rule of Eqs. 2-8 and
 * Sec. 2.4 (Arrhenius, equilibrium constant, third-body and Lindemann/Troe factors).
 * Arrays are device pointers of the precision's element type (CHEM_FP64: double,
 * CHEM_FP32: float; CHEM_SPLIT_BF16 returns CHEM_EUNSUPPORTED).  T[n], lnC[n][ldC].
 * Asynchronous on `stream`; argument errors are synchronous (CHEM_EINVAL).
 *
 * chem_source_term_jvp: domega[n][ldO] = d omega/dT * dT + d omega/d ln C * dlnC for a
 *   tangent dT[n], dlnC[n][ldC]; also omega[n][ldO] when omega is not NULL.
 * chem_source_term_vjp: g_T[n] = sum_k g_omega_k d omega_k/dT and
 *   g_lnC[n][ldC] = sum_k g_omega_k d omega_k/d ln C for a cotangent g_omega[n][ldG].
 * chem_source_term_jacobian: the dense Jacobian, cell index fastest:
 *   J[(k (n_species + 1) + m) ldJ + i] = d omega_k / d ln C_m of cell i for m < n_species,
 *   and d omega_k / dT for m = n_species; ldJ >= n_cells.
 */
chem_status chem_source_term_jvp(const chem_mech *mech, int64_t n_cells, const void *T,
                                 const void *lnC, int64_t ldC, const void *dT, const void *dlnC,
                                 void *omega, void *domega, int64_t ldO, chem_precision precision,
                                 void *stream);
chem_status chem_source_term_vjp(const chem_mech *mech, int64_t n_cells, const void *T,
                                 const void *lnC, int64_t ldC, const void *g_omega, int64_t ldG,
                                 void *g_T, void *g_lnC, chem_precision precision, void *stream);
chem_status chem_source_term_jacobian(const chem_mech *mech, int64_t n_cells, const void *T,
                                      const void *lnC, int64_t ldC, void *J, int64_t ldJ,
                                      chem_precision precision, void *stream);

/*
 * Exact equilibrium constants: lnKc[i * ldK + j] = ln K_c of reaction j at T[i] (Eqs. 8-11,
 * the Gibbs layer folded through the net stoichiometry in FP64 at load), FP64 device arrays,
 * ldK >= n_reactions.  The training targets of the approximate network below.
 * Asynchronous on `stream`.  Errors: CHEM_EINVAL, CHEM_ECUDA.
 */
chem_status chem_log_kc(const chem_mech *mech, int64_t n, const double *T, double *lnKc,
                        int64_t ldK, void *stream);

/*
 * Approximate-ANN equilibrium constants (Sec. 2.3, Eqs. 12-14; the paper's "Arch 2": the
 * only input is ln T).  x = (ln T - x_mean) / x_std; a_1 = act(w_in x + b_in);
 * a_{l+1} = act(W_l a_l + b_l) for l = 1 .. n_layers - 1; ln K_c,j = y_mean_j + y_std_j
 * (w_out,j . a + b_out,j).  All arrays are HOST float arrays copied by chem_kc_ann_load:
 * w_in, b_in [n_hidden]; w_hid [n_layers - 1][n_hidden][n_hidden] (row: output unit) and
 * b_hid [n_layers - 1][n_hidden] (may be NULL for one layer); w_out [n_reactions][n_hidden],
 * b_out, y_mean, y_std [n_reactions].  n_hidden <= 32.
 */
enum { CHEM_ACT_RELU = 0, CHEM_ACT_ELU = 1 };
typedef struct {
    int32_t n_layers, n_hidden, activation;
    float x_mean, x_std;
    const float *w_in, *b_in, *w_hid, *b_hid, *w_out, *b_out, *y_mean, *y_std;
} chem_kc_ann_desc;
typedef struct chem_kc_ann chem_kc_ann;       /* opaque, device-resident, immutable */

chem_status chem_kc_ann_load(const chem_mech *mech, const chem_kc_ann_desc *desc,
                             chem_kc_ann **out);
chem_status chem_kc_ann_free(chem_kc_ann *ann);

/*
 * The FP32 source term (float arrays, chem_source_term's layouts) with ln K_c of every
 * reversible reaction taken from the network instead of the Gibbs layer: an approximation
 * (its error is the network's), evaluated once per cell before the reaction loop.  It runs
 * the warp-per-cell FP32 kernel (one warp per cell, lanes over reactions).  ann == NULL
 * runs that same kernel with the exact Gibbs layer: the reference against which the
 * network's speed-up is measured (chem_source_term's CHEM_FP32 path may use another
 * kernel).  Errors: as chem_source_term, plus CHEM_EINVAL for a network of another
 * mechanism.
 */
chem_status chem_source_term_kc_ann(const chem_mech *mech, const chem_kc_ann *ann,
                                    int64_t n_cells, const float *T, const float *P,
                                    const float *Y, int64_t ldY, float *omega, int64_t ldO,
                                    void *stream);

/*
 * Constant-pressure adiabatic 0-D reactor: the stiff time integration the paper names as
 * future work for the source term (Conclusion; its own test integrates the same reactor
 * explicitly, Sec. 3.1.2).  Per cell the state is y = (T, Y_1 .. Y_ns) at fixed P and
 *   dY_k/dt = W_k omega_k / rho,        dT/dt = -sum_k H_k omega_k / (rho c_p)
 * with rho = P / (R T sum_k Y_k/W_k), C_k = rho Y_k / W_k, molar enthalpies
 * H_k = R T (h/RT)_k and c_p = sum_k Y_k R (cp/R)_k / W_k from the NASA-7 polynomials
 * (Eq. 10).  omega is Eqs. 2-11 and Sec. 2.4 with the mass-action products taken as
 * polynomials in C: negative mass fractions are NOT clipped here, so that the right-hand
 * side is smooth for an implicit integrator.  All arrays are FP64 DEVICE arrays;
 * T[n], P[n], Y[n][ldY].  Each cell is handled by one warp; results do not depend on the
 * other cells of the batch.
 *
 * chem_ode_rhs: f[i * ldF + 0] = dT/dt, f[i * ldF + 1 + k] = dY_k/dt; ldF >= n_species + 1.
 * chem_ode_jacobian: the analytic Jacobian, cell-major and row-major per cell:
 *   J[(i (n_species + 1) + r) (n_species + 1) + c] = d f_r / d y_c (index 0 is T).
 * Both are asynchronous on `stream`.  Errors: CHEM_EINVAL (NULL pointers with n > 0, n < 0,
 * ldY < n_species, ldF < n_species + 1, other device), CHEM_EUNSUPPORTED (a reaction with
 * more than 16 distinct species, or a mechanism whose per-warp vectors exceed shared
 * memory), CHEM_ENOMEM, CHEM_ECUDA.
 */
chem_status chem_ode_rhs(const chem_mech *mech, int64_t n_cells, const double *T,
                         const double *P, const double *Y, int64_t ldY, double *f,
                         int64_t ldF, void *stream);
chem_status chem_ode_jacobian(const chem_mech *mech, int64_t n_cells, const double *T,
                              const double *P, const double *Y, int64_t ldY, double *J,
                              void *stream);

/* Per-cell outcome of chem_integrate_cells. */
enum { CHEM_CELL_OK = 0, CHEM_CELL_STEP_UNDERFLOW = 1, CHEM_CELL_MAX_STEPS = 2,
       CHEM_CELL_NONFINITE = 3 };

/* Options of chem_integrate_cells; a NULL pointer means all defaults. */
typedef struct {
    double h_init;          /* first step (s); <= 0: automatic, 0.01 |y| / |f(y0)| in the
                               error norm's weighted RMS, at most t_end */
    double h_min;           /* a cell fails when its step falls below this (s); <= 0: only
                               when a step no longer advances t in double precision */
    double h_max;           /* largest step (s); <= 0: t_end */
    int64_t max_steps;      /* attempted steps per cell before it fails; <= 0: 100000 */
    double ign_dT;          /* ignition event: first time T reaches T0 + ign_dT; <= 0: 400 K */
    double *t_ign;          /* [n] device or NULL: ignition time (s), linear in T within the
                               accepted step that crosses; -1 when not reached */
    int32_t *n_accepted;    /* [n] device or NULL: accepted steps per cell */
    int32_t *n_rejected;    /* [n] device or NULL: rejected steps per cell */
    int32_t fixed_steps;    /* > 0: take exactly this many equal steps of t_end / fixed_steps
                               with no error control (every step accepted; a cell whose state
                               stops being finite gets CHEM_CELL_NONFINITE); 0: adaptive */
    int32_t jacobian_fp32;  /* nonzero: the stage Jacobian in FP32 (Rodas3's order assumes the
                               exact Jacobian; measured 11 % more steps/s at 53/325); 0: FP64.
                               The right-hand side, LU, solves and error control are FP64 */
} chem_integrate_opts;

/*
 * Integrate every cell's reactor from t = 0 to t_end in place: on return T[n] and
 * Y[n][ldY] hold the state at t_end (P[n] is constant).  Rosenbrock method Rodas3
 * (Sandu et al. 1997: four stages, order 3 with an embedded order-2 solution, stiffly
 * accurate and L-stable) with the analytic Jacobian of chem_ode_jacobian, an FP64 LU with
 * partial pivoting per step, and per-cell step-size control on the RMS norm of the
 * embedded error with weights atol + rtol max(|y_old|, |y_new|); each cell takes its own
 * steps, so its result does not depend on the rest of the batch.  cell_status[n] (device,
 * may be NULL) receives CHEM_CELL_*; a failed cell keeps its last accepted state.
 * The call allocates a small device workspace on `stream` (stream-ordered) and
 * SYNCHRONISES `stream` before returning, to report failures: CHEM_ENONCONV when at
 * least one cell failed (the others are valid).  Errors: as chem_ode_rhs, plus
 * CHEM_EINVAL for t_end < 0, rtol <= 0 or atol < 0.
 */
chem_status chem_integrate_cells(const chem_mech *mech, int64_t n_cells, double *T,
                                 const double *P, double *Y, int64_t ldY, double t_end,
                                 double rtol, double atol, const chem_integrate_opts *opts,
                                 int32_t *cell_status, void *stream);

/*
 * chem_integrate_cells without any allocation (the paper has no counterpart: this is a
 * deployment variant).  Same arguments, semantics, synchronisation and errors as
 * chem_integrate_cells, but the device workspace comes from a static 1 MiB array per
 * device instead of a stream-ordered allocation, for callers that cannot let the library
 * allocate (device memory handed to a CFD solver's or framework's own pool allocator, or a
 * time-step loop that must not pay an allocation's latency or implicit synchronisation).
 * The array is shared by all calls on a device: calls that overlap in time on one device
 * race on it and must not be issued.  Each call clears the part that must start at zero
 * (cell counter, failure count) on its stream, and looks up the array's address on the
 * current device (no allocation).  The first call on a device may load the module that
 * holds the array; make it before any stream capture on that device.
 * Additional error: CHEM_ENOMEM for a mechanism whose reactor matrices do not fit in
 * shared memory (they would need per-warp matrices in device memory), whatever n_cells is.
 */
chem_status chem_integrate_cells_noalloc(const chem_mech *mech, int64_t n_cells, double *T,
                                         const double *P, double *Y, int64_t ldY, double t_end,
                                         double rtol, double atol,
                                         const chem_integrate_opts *opts, int32_t *cell_status,
                                         void *stream);

/*
 * The classical coefficients of the integrator's Rosenbrock method (host call, no GPU
 * needed): *stages = s, gamma_ii = *gamma, alpha[s][s] and gamma[s][s] strictly lower
 * (row-major, 4 x 4 buffers), b[s] and the embedded bhat[s], in the form
 *   (I - h gamma_ii J) k_i = h f(y + sum_j alpha_ij k_j) + h J sum_j gamma_ij k_j,
 *   y_new = y + sum_i b_i k_i.
 */
chem_status chem_rosenbrock_tableau(int32_t *stages, double *gamma_ii, double *alpha,
                                    double *gamma, double *b, double *bhat);

/*
 * Serving: a persistent request loop for many producers (the paper's offload pattern, in
 * which every CFD rank hands its cells to the GPU for the source term, Secs. 1 and 3.2).
 * A server owns one host worker thread, four streams ("lanes"), one device block of the
 * HBM budget with a page-locked host mirror of the same size, and the CUDA graphs it has
 * captured.  submit() only queues; when a lane is free the worker packs the oldest queued
 * request that lane may run, with later queued requests that share (mechanism, kind,
 * precision, dt, tolerances), into one batch, takes the batch's bytes from the budget
 * (first fit), copies the batch to the device, replays the lane's graph for that key
 * (updated in place with the batch's pointers and cell count) and copies the results back,
 * while other lanes' batches run: requests that arrive while the GPU is busy are admitted
 * as soon as a lane and enough of the budget are free; a request that does not fit yet
 * waits for a batch to retire.  The SMs are split in two partitions (green contexts where
 * the driver provides them, else by the persistent kernels' grid sizes): 16 SMs for lanes
 * 0 and 1, which take source-term batches only, and the rest for lanes 2 and 3, which take
 * integrations (and source-term batches while no integration is queued or running), so
 * that source-term requests do not wait behind long integrations.  A source-term batch
 * holds at most 2^20 cells and an integration batch at most 65536 (a larger single request
 * runs alone).  Cells are independent, so a request's result does not depend on the batch
 * it ran in.
 * The mechanisms must outlive the server.  All calls are thread-safe.
 */
enum { CHEM_REQ_SOURCE = 0, CHEM_REQ_INTEGRATE = 1 };

typedef struct {
    int32_t mech_index;         /* index into the server's mechanism list */
    int32_t kind;               /* CHEM_REQ_SOURCE or CHEM_REQ_INTEGRATE */
    chem_precision precision;   /* SOURCE: element type of T, P, Y, omega (CHEM_FP64: double,
                                   otherwise float); INTEGRATE: must be CHEM_FP64 */
    int32_t fixed_steps;        /* INTEGRATE: 0 adaptive over dt; k > 0: k equal steps of dt / k
                                   without error control (chem_integrate_opts.fixed_steps) */
    int64_t n_cells;            /* >= 1 */
    const void *T, *P, *Y;      /* HOST arrays [n], [n], [n][n_species] (dense rows) */
    void *omega;                /* SOURCE: HOST output [n][n_species] */
    double *T_out, *Y_out;      /* INTEGRATE: HOST outputs [n], [n][n_species]; may alias T, Y */
    int32_t *cell_status;       /* INTEGRATE: HOST output [n] (CHEM_CELL_*), or NULL */
    double dt, rtol, atol;      /* INTEGRATE: time to advance (s) and tolerances */
} chem_request;

typedef struct {
    chem_status status;         /* of the request's batch; CHEM_ENONCONV: some cell failed */
    int32_t batch_requests;     /* requests in the batch it ran in */
    int64_t n_cells;
    int64_t batch_cells;        /* cells of that batch */
    int32_t n_failed;           /* INTEGRATE: cells with a nonzero status */
    int32_t slot;               /* lane the batch ran on */
    double queue_us;            /* submit -> batch launch */
    double latency_us;          /* submit -> results in the caller's host arrays */
    int64_t steps_accepted;     /* INTEGRATE: accepted steps summed over the request's cells */
    int64_t steps_rejected;     /* INTEGRATE: rejected steps summed over its cells */
} chem_result;

typedef struct {
    int32_t n_slots;            /* lanes (streams) */
    int64_t slot_cells;         /* most cells of one source-term batch */
    size_t device_bytes;        /* device memory the server holds (the budget) */
    uint64_t submitted, completed, batches, graphs_captured, graph_launches;
    int32_t max_batch_requests; /* most requests seen in one batch */
    uint64_t graph_updates;     /* launches whose cached graph was updated in place */
    uint64_t memory_waits;      /* requests that waited for part of the budget to free up */
    size_t bytes_in_use;        /* budget held by batches in flight now */
    size_t bytes_in_use_max;    /* and the most held at once */
    int32_t source_sms;         /* SMs of the source-term partition (lanes 0, 1) */
    int32_t integrate_sms;      /* SMs of the integration partition (lanes 2, 3) */
    int32_t green_contexts;     /* 1: partitions are green contexts; 0: kernel grids only */
} chem_serve_info;

/*
 * Create a server for n_mechs loaded mechanisms (same device) holding hbm_budget bytes of
 * device memory (one allocation, carved per batch) and as much page-locked host memory.
 * Errors: CHEM_EINVAL, CHEM_ENOMEM (budget below one batch of 64 cells of the largest
 * mechanism, or an allocation failed), CHEM_ECUDA.
 */
chem_status chem_serve_create(const chem_mech *const *mechs, int32_t n_mechs, size_t hbm_budget,
                              void **server);

/*
 * Queue a request without blocking; *ticket identifies it.  The host arrays must stay valid
 * until chem_serve_poll reports the request complete.  Errors, synchronous: CHEM_EINVAL
 * (malformed request), CHEM_ENOMEM (the request alone needs more than the whole budget),
 * CHEM_EUNSUPPORTED (a path this mechanism does not support), CHEM_EBUSY (server stopping).
 */
chem_status chem_serve_submit(void *server, const chem_request *req, uint64_t *ticket);

/*
 * Wait up to timeout_us (0: do not wait; < 0: wait without limit) for a ticket.  On
 * completion fills *result, releases the ticket and returns CHEM_OK (the request's own
 * outcome is result->status).  CHEM_ENOTREADY: timeout_us == 0 and not done;
 * CHEM_ETIMEOUT: the wait ran out; CHEM_EINVAL: unknown or already released ticket.
 */
chem_status chem_serve_poll(void *server, uint64_t ticket, chem_result *result,
                            int64_t timeout_us);

/* Counters of a server. */
chem_status chem_serve_info_get(void *server, chem_serve_info *info);

/* Stop the worker after the batches on the GPU finish, release everything.  Requests still
 * queued are dropped; their tickets become invalid. */
chem_status chem_serve_destroy(void *server);

/*
 * Device-side status of a mechanism's tensor-core kernels.  Every wait inside them is
 * bounded; a kernel that gives up records a nonzero code (1 tile loader, 2 MMA issuer,
 * 3 epilogue) and its output is then invalid.  This call synchronises the current
 * device, returns the code in *code (0: no failure since the last query) and clears it.
 */
chem_status chem_device_status(const chem_mech *mech, int32_t *code);

/* Number of kernels this library has launched in the process so far. */
uint64_t chem_kernel_launch_count(void);

/* Message of the last failed call on the calling thread ("" if none). */
const char *chem_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CHEM_H */
