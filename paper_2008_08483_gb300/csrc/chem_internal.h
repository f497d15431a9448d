// chem_internal.h -- device table layouts and shared declarations of the library.
// Included by the library's own translation units only.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>

#include "chem.h"

namespace chem {

constexpr int kMaxSide = 8;                       // species per reaction side (SIMT tables)
constexpr int kMaxSpecies = 1024;
constexpr int kMaxReactions = 65536;
constexpr double kR = 8.31446261815324e7;         // erg / (mol K)
constexpr double kLog2e = 1.44269504088896340736;
constexpr double kLn2 = 0.69314718055994530942;

// One reaction for the FP64 paths (source term, derivatives, reactor).  Natural-log units.
// The source-term kernel reads it from a slot-major copy (MechViewF64::rxn_t).
struct alignas(16) RxnF64 {
    double lnA, b, EoR;          // ln k_inf = lnA + b ln T - EoR / T            (Eq. 6)
    double kc[2][7];             // ln K_c per T range on [1, ln T, tau, tau^2, tau^3, tau^4, 1/T],
                                 // tau = T / 1000, folded from NASA-7 through nu (Eqs. 9-11)
    double low[3];               // ln k0 = low0 + low1 ln T - low2 / T           (falloff)
    double troe[5];              // 1 - alpha, alpha, 1/T***, 1/T*, T** (<= 0: absent)
    int32_t kind, rev;
    int32_t tb_begin, tb_end;    // third-body list range (kinds 1-3)
    int32_t nf, nr;              // species on each side
    uint16_t spf[kMaxSide], spr[kMaxSide];
    uint8_t nuf[kMaxSide], nur[kMaxSide];
};

// One reaction for the FP32 SIMT path.  log2 units; double-float (hi, lo) coefficients
// for the large-magnitude parts of the exponent.
struct alignas(16) RxnF32 {
    float2 kf[3];                // log2 k_inf on [1, log2 T, 1/T]
    float2 k0[3];                // log2 k0 on [1, log2 T, 1/T]
    float troe[5];               // 1 - alpha, alpha, 1/T***, 1/T*, T**
    int32_t kind, rev;
    int32_t tb_begin, tb_end;
    int32_t nf, nr, dnu;         // dnu = sum_k nu_kj
    int32_t ordf, ordr;          // reaction orders sum nu', sum nu''
    uint16_t spf[kMaxSide], spr[kMaxSide];
    uint8_t nuf[kMaxSide], nur[kMaxSide];
};

// Per species: -g_k/(RT) in log2 units on [1, log2 T, tau, tau^2, tau^3, tau^4, 1/T] as
// double-float pairs, for each T range (FP32 path Gibbs layer, Eq. 10).
struct alignas(16) SpecF32 {
    float2 gl[2][7];
    float invW;
    float pad[3];
};

// One reaction for the reactor integrator: the distinct species of the reaction as Jacobian
// rows (net coefficient nu''_k - nu'_k != 0) and columns (any species on either side, with
// its nu' and nu''), so that the per-reaction updates of omega and of d omega / dC touch
// distinct entries.
constexpr int kIntMax = 16;
struct alignas(16) RxnInt {
    int32_t nrow, ncol;
    uint16_t row_sp[kIntMax];
    uint16_t col_sp[kIntMax];
    uint8_t col_nuf[kIntMax], col_nur[kIntMax];
    double row_nu[kIntMax];      // nu''_k - nu'_k
};

struct IntView {
    const RxnInt *rxn;
    const int32_t *order;        // [n_slots] reaction processing order, -1 = empty slot;
                                 // grouped by kind in blocks of 32 (warp-uniform kind)
    int32_t n_slots;
    // per group of 32 slots, the reactions of the group that change species k:
    // entries gptr[g (ns + 1) + k] .. gptr[g (ns + 1) + k + 1] of (slot, nu''_k - nu'_k)
    const int32_t *gptr;
    const int32_t *gent_slot;
    const double *gent_nu;
    const double *nasa;          // [ns][2][7] NASA-7 sets (T < t_mid, T >= t_mid)
    const double *W;             // [ns] molecular weights
    bool ok;                     // every reaction fits kIntMax
};

struct MechViewF64 {
    int ns, nr;
    const RxnF64 *rxn;
    const uint16_t *tb_sp;       // third-body species lists
    const double *tb_e;          // efficiency - 1 for listed species
    const double *invW;          // [ns] 1 / W_k
    double t_mid;
    // as in MechViewF32: the records as slot-major 32-bit words (kind-grouped slots) and the
    // species-major net stoichiometry with its species-to-lane schedule (shared arrays)
    const uint32_t *rxn_t;
    int32_t n_slots;
    const int32_t *col_ptr, *col_rxn;
    const float *col_nu;
    const int32_t *lane_ptr, *lane_sp;
    // species-major reaction sides (nu', nu'' of each reaction on which species k appears)
    // and listed third-body efficiencies (eff - 1), for the vjp gather
    const int32_t *sd_ptr, *sd_rxn;
    const float *sd_nuf, *sd_nur;
    const int32_t *ts_ptr, *ts_rxn;
    const double *ts_e;
};

// Approximate-ANN ln K_c (Sec. 2.3, Eqs. 12-14): standardised ln T -> N_L hidden layers of
// N_H units (ReLU or ELU) -> N_R standardised ln K_c, all weights FP32 in device memory.
constexpr int kAnnMaxHidden = 32;
struct KcAnnView {
    int nl, nh, act;             // act: 0 ReLU, 1 ELU
    float x_mean, x_inv_std;
    const float *w_in, *b_in;    // [nh], [nh]
    const float *w_hid, *b_hid;  // [nl-1][nh][nh] (input-major: [input][output]), [nl-1][nh]
    const float *w_out, *b_out;  // [nh][nr] (hidden-unit-major), [nr]
    const float *y_mean, *y_std; // [nr]
};

struct MechViewF32 {
    int ns, nr;
    const SpecF32 *spec;
    const uint16_t *tb_sp;
    const float *tb_e;
    float t_mid;
    float2 lg2_pref_R;           // log2(p_ref / R), double-float
    // species-major net stoichiometry (Eq. 2 as a gather): the reactions that change species
    // k are entries col_ptr[k] .. col_ptr[k + 1] of (col_rxn, col_nu = nu''_kj - nu'_kj),
    // in reaction order
    const int32_t *col_ptr;
    const int32_t *col_rxn;
    const float *col_nu;
    // the gather's species per lane, balanced by entry count: lane l takes species
    // lane_sp[lane_ptr[l]] .. lane_sp[lane_ptr[l + 1] - 1]
    const int32_t *lane_ptr;
    const int32_t *lane_sp;
    // the reaction records as 32-bit words, slot-major ([word][slot], slots in the kind-
    // grouped processing order, empty slots zero), so that 32 lanes reading one field of 32
    // consecutive slots make one coalesced load
    const uint32_t *rxn_t;
    int32_t n_slots;
};

// Tables of the thread-per-cell FP32 kernel (kern_f32t.cu).  Exponents are kept as a head H
// on the grid of multiples of 2^-12 (sums of heads are exact in FP32) and a small remainder L.
// Temperature terms are centred on T0 = 1000 K: d1 = log2 T - log2 T0, d2 = 1/T - 1/T0.
// A reaction record of the kernel (128 bytes).  Entries are (byte offset of the species' row
// in the warp's shared tables, coefficient as float bits) pairs, in the order
//   reactant 0, 1 | product 0, 1 | net 0, 1 | net 2, 3 | reactant 2, product 2 | net 4, 5
// so that a reaction with at most two species per side reads six 16-byte words; unused
// entries point at a zero row past the last species with coefficient 0.
constexpr int kTSide = 3;                 // reactant and product slots per reaction
constexpr int kTNet = 6;                  // net-change slots per reaction
struct alignas(16) RxnT {
    float4 kf;                   // log2 k_inf(T0) as (H, L); coefficient of d2 (-E/R log2 e)
                                 // as double-float (hi, lo)
    float b;                     // coefficient of d1 (temperature exponent)
    uint32_t meta;               // group type | falloff index << 8
    uint32_t tb;                 // first record of a quad: its efficiency lists in the
                                 // staged table, first | entries per reaction << 16
    float rb;                    // added to the reverse exponent: 0, or -2000 if irreversible
    int32_t ent[24];
};
__host__ __device__ constexpr int rxnt_react(int s) { return s < 2 ? s : 8; }
__host__ __device__ constexpr int rxnt_prod(int s) { return s < 2 ? 2 + s : 9; }
__host__ __device__ constexpr int rxnt_net(int s) { return s < 4 ? 4 + s : 6 + s; }
// Per falloff reaction: low-pressure limit as kf; (b0, 1 - alpha, alpha, -log2 e / T***);
// (-log2 e / T*, -T** log2 e, 1 if the T** term is present else 0, 0)
struct alignas(16) FallT {
    float4 k0;
    float4 t0;
    float4 t1;
};
struct alignas(16) SpecT {
    float4 ga[2];                // per T range: G(T0) as (H, L); coefficient of d1 (hi, lo)
    float4 gb[2];                // coefficient of d2 (hi, lo); e1, e2 of the centred polynomial
    float4 gc[2];                // e3, e4; 1 / W_k; 0
};
struct F32TView {
    int ns, n_rec;               // species; records (groups padded to pairs)
    int n_tb, n_fall;
    const RxnT *rxn;
    const SpecT *spec;
    const int2 *tb;              // (row offset, efficiency - 1 as float bits)
    const FallT *fall;
    double t_mid;
    // double-float (hi, lo) constants: log2 T0, 1/T0, log2 R, log2(p_ref / R), log2 e
    float2 lg2T0, invT0, lg2R, lg2_pref_R, log2e;
    float Tc[2];                 // centre (K) of each T range's Gibbs polynomial
    bool ok;                     // the mechanism fits the kernel (else the warp-per-cell kernel)
};

}  // namespace chem

// The opaque handle of the C ABI.
struct chem_mech {
    int ns, nr, device;
    double t_mid, p_ref;
    size_t device_bytes;
    void *d_blob;
    chem::MechViewF64 v64;
    chem::MechViewF32 v32;
    chem::IntView vint;
    chem::F32TView vt;           // thread-per-cell FP32 tables (vt.ok false: not built)
    void *d_f32t;
    bool have_bf16;
    bool bf16_wide;              // the tables are those of the large-mechanism kernel
    void *bf16;                  // split-BF16 tables (tensor-core path): kern_bf16.cu, or
                                 // kern_wide.cu when bf16_wide
    // resident warps of the SIMT source-term kernels on the mechanism's device (0: not yet
    // queried): FP64, FP32, FP32 with the ln K_c network
    std::atomic<int> simt_warps[3];
};

namespace chem {

chem_status set_error(chem_status st, const char *fmt, ...);

// Opt-in of a kernel to more than the default dynamic shared memory on the current device,
// cached per device.  The attribute lives in the device's context, which cudaDeviceReset
// discards; a launcher whose launch fails therefore calls ensure(..., true) and retries
// once (launch_opted).
struct SmemOptIn {
    std::atomic<uint64_t> done{0};
    chem_status ensure(const void *func, int bytes, bool force, const char *name)
    {
        int dev = 0;
        cudaGetDevice(&dev);
        const uint64_t bit = 1ull << (dev & 63);
        if (!force && (done.load() & bit)) return CHEM_OK;
        cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) return set_error(CHEM_ECUDA, "%s attribute: %s", name, cudaGetErrorString(e));
        done.fetch_or(bit);
        return CHEM_OK;
    }
};

// Launch through `launch` (a callable doing the <<<>>> launch) after the opt-in; on a
// launch error, opt in again and retry once.
template <class F>
chem_status launch_opted(SmemOptIn &opt, const void *func, int bytes, const char *name, F &&launch)
{
    for (int attempt = 0; attempt < 2; ++attempt) {
        chem_status st = opt.ensure(func, bytes, attempt > 0, name);
        if (st != CHEM_OK) return st;
        launch();
        const cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) return CHEM_OK;
        if (attempt > 0) return set_error(CHEM_ECUDA, "%s launch: %s", name, cudaGetErrorString(e));
    }
    return CHEM_OK;
}
// ln K_c of reaction j in temperature range r on [1, ln T, tau, tau^2, tau^3, tau^4, 1/T]
void fold_kc(const chem_mech_desc *d, int j, int r, double out[7]);
void clear_error();
extern std::atomic<uint64_t> g_launches;
// Most SMs a persistent kernel's grid covers when launched from the calling thread (0: all
// of the device).  The serving worker sets it while it records a batch for an SM partition.
extern thread_local int tl_sm_limit;
inline int sm_limit(int nsm) { return tl_sm_limit > 0 && tl_sm_limit < nsm ? tl_sm_limit : nsm; }

// Reactor integration without allocation or synchronisation (kern_integrate.cu): the
// workspace size for up to n_max cells, the argument checks of chem_integrate_cells, and the
// launch itself (header clear + persistent kernel; n_dev optionally holds the cell count).
size_t integrate_workspace_bytes(const chem_mech *m, int64_t n_max);
size_t integrate_header_bytes();   // the part of the workspace that does not grow with n
chem_status integrate_checks(const chem_mech *m, int64_t n, const double *T, const double *P,
                             const double *Y, int64_t ldY, double t_end, double rtol, double atol);
chem_status integrate_launch(const chem_mech *m, int64_t n_max, const int64_t *n_dev, double *T,
                             const double *P, double *Y, int64_t ldY, double t_end, double rtol,
                             double atol, const chem_integrate_opts *opts, int32_t *cell_status,
                             void *ws, size_t ws_bytes, cudaStream_t s);

chem_status launch_source_fp64(const chem_mech *m, int64_t n, const double *T, const double *P,
                               const double *Y, int64_t ldY, double *om, int64_t ldO,
                               cudaStream_t s);
chem_status launch_source_fp32(const chem_mech *m, int64_t n, const float *T, const float *P,
                               const float *Y, int64_t ldY, float *om, int64_t ldO,
                               cudaStream_t s);
// the warp-per-cell FP32 kernel with the exact Gibbs layer, whatever the mechanism's size
// (the structure the network variant shares)
chem_status launch_source_fp32_warp(const chem_mech *m, int64_t n, const float *T, const float *P,
                                    const float *Y, int64_t ldY, float *om, int64_t ldO,
                                    cudaStream_t s);
chem_status launch_source_fp32_ann(const chem_mech *m, const KcAnnView &av, int64_t n,
                                   const float *T, const float *P, const float *Y, int64_t ldY,
                                   float *om, int64_t ldO, cudaStream_t s);
chem_status launch_log_kc(const chem_mech *m, int64_t n, const double *T, double *lnkc,
                          int64_t ldK, cudaStream_t s);

// Thread-per-cell FP32 source term (kern_f32t.cu): tables built at load (a mechanism the
// kernel does not take leaves m->vt.ok false) and the launch, used by launch_source_fp32.
chem_status f32t_build_tables(chem_mech *m, const chem_mech_desc *d);
void f32t_free_tables(chem_mech *m);
chem_status launch_source_fp32_t(const chem_mech *m, int64_t n, const float *T, const float *P,
                                 const float *Y, int64_t ldY, float *om, int64_t ldO,
                                 cudaStream_t s);

}  // namespace chem
