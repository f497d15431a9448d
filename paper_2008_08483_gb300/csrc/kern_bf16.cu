// kern_bf16.cu -- split-BF16 source term on tcgen05 tensor cores (sm_103a).
//
// Per tile of 128 cells (one cell per tensor-memory lane), for reaction chunks of RC = 64:
//   contraction 1 (Eqs. 4, 11): S = log2 X . [nu' | nu''] (M=128, N=2 RC=128, K=NSP), and
//       the reverse half also accumulates G . nu, the Gibbs layer of Eq. 11 (G_k = g_k/(RT)
//       log2 e - log2(p_ref/(RT)), per cell and species, three BF16 terms in tensor memory;
//       nu is contraction 2's table read as an MN-major operand), so that S'' + log2 k_f =
//       sum_k nu''_k log2 C_k + log2 k_r
//       A = log2 X in tensor memory as three BF16 terms (hi + mid + lo); the extra
//       column NSP_extra = log2 c_tot carries the reaction orders (and the third-body
//       c_tot factor), so S = sum_k nu_k log2 C_k (+ log2 c_tot for third-body).
//       B = the small-integer stoichiometric matrices, exact in BF16, in shared memory.
//       When nine padding columns are free (NSP >= ns + 11), they carry the Arrhenius layer
//       (Eq. 6) as well: features [1, log2 T, 1/T] (three BF16 terms each) against the
//       coefficients [log2 A, b, -E/R log2 e] (three BF16 rows each), so that S' = log2 q_f and
//       S'' = log2 q_r directly; an irreversible reaction's reverse column and an empty slot
//       carry a bias of -1e4 (2^S = 0).
//   epilogue (FP32, one thread per cell): without the folded Arrhenius layer, log2 k_f
//       (Eq. 6) added to both halves; third-body / falloff factors (Sec. 2.4),
//       q = 2^S' - 2^S'', q_net = q_f - q_r (Eq. 3), split into two BF16 terms written to
//       tensor memory.
//   contraction 2 (Eq. 2):  omega += q_net . nu^T          (M=128, N=NSP, K=RC)
//   contraction 0 (Sec. 2.4), once per tile, issued after chunk 0's contraction 1 (before
//       it when chunk 0 itself reads multipliers): the third-body sums
//       sum_k (eff_jk - 1) z_k of the reactions that need them (M=128, N=64, K=NSP), A = z as
//       two BF16 terms in contraction 2's operand columns (free until chunk 0's q_net), B =
//       eff - 1 as two BF16 terms (hi.hi + hi.lo + lo.hi), into the multiplier columns.
// omega accumulates in tensor memory across the chunks and is written once per tile.
// Contraction 1 of chunk c + 1 runs while the epilogue works on chunk c (it starts as soon
// as chunk c's S has been read out), contraction 2 of chunk c as soon as its q_net is in.
//
// Tiles overlap: the next tile's prologue runs as soon as every contraction 1 of the current
// tile has completed (A1FREE), before the current tile's omega is read out of tensor memory
// and stored, so that the next tile's contraction 1 starts meanwhile.
// Warp roles (608 threads): warp 0 bulk-copies the T, P, Y tile into shared memory;
// warp 1 owns tensor memory and issues contractions 0 and 1 from one thread, warp 18
// contraction 2 (an MMA issue blocks while the tensor pipe is busy, so one issuer would sit
// on contraction 2 of chunk c while chunk c + 1's S has been read out); warps 2-17 form four
// epilogue warpgroups, warpgroup g taking reactions 16 g .. 16 g + 15 of every chunk (warp
// w reaches tensor-memory lanes 32 (w % 4) .. 32 (w % 4) + 31).  Reactions with a third-body
// or falloff factor sit in the first 8 slots of the last chunks' quarters (falloff ones in
// slots 0..3); the epilogue turns contraction 0's sums into M / c_tot and, for the falloff
// slots, into Pr / (1 + Pr) F where the quarter's rates are formed.
// Every mbarrier wait is bounded: on timeout the kernel records an error code in the
// mechanism's device status word and all roles wind down.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "chem_internal.h"
#include "tc_ptx.h"

namespace chem {

constexpr int RC = 64;                 // reactions per chunk
constexpr int RH = RC / 4;             // reactions per warpgroup and chunk
constexpr int NQ = RC / RH;            // warpgroups (chunk quarters)
constexpr int kEpiWarp0 = 2;           // first epilogue warp
constexpr int kEpiWarps = 16;
constexpr int kMma2Warp = kEpiWarp0 + kEpiWarps;   // issues contraction 2
constexpr int kThreads = 32 * (kMma2Warp + 1);
constexpr uint32_t kTmemCols = 512;
constexpr float kLog2Floor = -1000.0f; // log2 X of an absent species: 2^x underflows to 0
constexpr float kDead = -1.0e4f;       // log2 of a rate constant that is zero
constexpr int kFoldRows = 9;           // K rows of the folded Arrhenius layer: 3 features x 3 terms

constexpr int kFacCols = 64;           // multiplier columns: 8 per quarter holding such reactions

// per-reaction coefficients, copied to shared memory with the stoichiometric tables (read by
// the epilogue when the Arrhenius layer is not folded into contraction 1)
struct alignas(16) CoefS {
    float4 kf;         // Arrhenius layer (Eq. 6): log2 k_inf = x + y log2 T + z / T;
                       // w = 1 for a reversible reaction, 0 otherwise (Sec. 2.4)
};
// per species: G_k = g_k/(RT) log2 e - log2(p_ref/(RT)) on [1, log2 T, tau, tau^2, tau^3,
// tau^4, 1/T] (tau = T/1000), one set per temperature range (Eq. 10 with the standard
// concentration folded into the bias as in Eq. 11)
struct alignas(16) GibbsS {
    float c[2][8];
};
// slot 0..3 of a chunk quarter holding third-body / falloff reactions: the falloff layer
// (Sec. 2.4), or neutral values with kf.w = 0 (the multiplier is then M / c_tot)
struct alignas(16) FallQ {
    float4 kf;         // log2 k_inf = x + y log2 T + z / T; w = 1 for a falloff reaction
    float4 k0;         // log2 k0 = x + y log2 T + z / T
    float4 troe;       // 1 - alpha, alpha, log2(e)/T***, log2(e)/T* (Lindemann: 1, 0, 0, 0)
    float4 t2;         // x = log2(e) T** (absent: 1e30, the term underflows to zero)
};

struct Bf16Tables {
    int nsp, nch, fac_chunk0;
    bool fold;                                   // Arrhenius layer folded into contraction 1
    size_t b1_bytes, blob_bytes;
    uint32_t o_b2, o_e, o_coef, o_hmask, o_fq, o_gib;   // offsets from the blob start
    void *d_blob;
    const uint16_t *btab;     // one contiguous block copied to shared memory
    const float *invW;
    int *status;
};

struct Bf16Params {
    const float *T, *P, *Y;
    float *om;
    int64_t n, ldY, ldO;
    int ns, nch, ntiles;
    int fac_chunk0;            // chunk 0 holds third-body / falloff reactions
    int stage_y;               // T, P, Y tiles staged in shared memory (the Y buffer then also
                               // stages omega on its way out)
    int bulk_out;              // omega rows contiguous (ldO == ns) and 16-byte aligned
    const uint16_t *btab;
    uint32_t blob_bytes;
    const float *invW;
    float t_mid, lg2R;
    int *status;
    // shared-memory layout (byte offsets from the 1024-aligned base); the copied block
    // holds B1, B2, the efficiency table, coefficients, quarter masks, falloff records and
    // the Gibbs layer
    uint32_t o_b2, o_e, o_coef, o_hmask, o_fq, o_gib, o_y, o_t, o_p, o_iw, o_psum, o_bar;
};

enum {
    BAR_BTAB, BAR_YFULL, BAR_YEMPTY, BAR_A1FULL, BAR_D1FULL, BAR_D1EMPTY, BAR_A2FULL, BAR_A2EMPTY,
    BAR_D2FULL, BAR_D2EMPTY, BAR_XREADY, BAR_A1FREE, BAR_DRAIN, BAR_WREADY, BAR_ZFREE, BAR_COUNT
};

struct SmemCtl {
    uint32_t tmem_base;
    volatile int abort;
    volatile int mma1_issued;   // contractions 1 issued so far (an ordering hint only)
};

// Bounded mbarrier wait: gives up after ~2^31 cycles (about a second), or as soon as
// another role has given up, recording `code` in the device status word.
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity, SmemCtl *ctl, int *status,
                                         int code)
{
    if (tc::mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (true) {
        if (tc::mbar_try_wait_sleep(bar, parity, 20000)) return true;
        if (ctl->abort) return false;
        if (clock64() - t0 > (1ll << 31)) {
            ctl->abort = 1;
            atomicCAS(status, 0, code);
            return false;
        }
    }
}

template <int NSP>
struct Cols {                                     // tensor-memory column map
    static constexpr uint32_t A1 = 0;             // log2 z: 3 splits x NSP/2 columns
    static constexpr uint32_t AG = ((3 * NSP / 2 + 31) / 32) * 32;   // G: 3 splits x NSP/2
    static constexpr uint32_t D1 = AG + ((3 * NSP / 2 + 31) / 32) * 32;   // 2 RC: S', S''
    static constexpr uint32_t A2 = D1 + 2 * RC;   // 2 splits x RC/2
    static constexpr uint32_t D2 = A2 + RC;       // NSP columns
    static constexpr uint32_t FC = D2 + NSP;      // third-body sums (contraction 0)
    static_assert(FC + kFacCols <= kTmemCols, "tensor memory over budget");
};

// Per-cell features kept in registers by every epilogue thread.
struct CellF {
    float lg2T, invT, tau, tau2, lgct, inv_sum;
    int rg;
};

// Shared-memory view of the per-reaction tables.
struct SmemTabs {
    const CoefS *coef;
    const uint32_t *hmask;     // per chunk quarter: nonzero if it holds third-body / falloff
                               // reactions (in its first 8 slots)
    const int *fbase;          // per chunk quarter: its first multiplier column (8 each)
    const FallQ *fq;           // per such quarter, slots 0..3
};

// Multipliers of q_net for slots 0..3 of a quarter holding third-body / falloff reactions
// (Sec. 2.4), from s = M / c_tot: Pr / (1 + Pr) F for a falloff reaction (F = 1 for
// Lindemann, the Troe form otherwise), s itself for the others.  Branch-free over the four
// slots so that their dependency chains interleave.
__device__ __forceinline__ void falloff4(const FallQ *F, const float (&s)[8], const CellF &c,
                                         float (&out)[4])
{
    const float Tn = c.tau * 1000.0f;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const float4 kf = F[u].kf, k0 = F[u].k0, tr = F[u].troe;
        const float t2 = F[u].t2.x;
        const float lkf = fmaf(kf.z, c.invT, fmaf(kf.y, c.lg2T, kf.x));
        const float lk0 = fmaf(k0.z, c.invT, fmaf(k0.y, c.lg2T, k0.x));
        const float lpr = lk0 - lkf + c.lgct + tc::lg2(fmaxf(s[u], 1e-30f));   // log2 Pr
        float fac = -tc::lg2(1.0f + tc::ex2(-lpr));               // log2(Pr / (1 + Pr))
        const float fc = tr.x * tc::ex2(-Tn * tr.z) + tr.y * tc::ex2(-Tn * tr.w) +
                         tc::ex2(-t2 * c.invT);
        const float lfc = tc::lg2(fc);                             // log2 F_cent
        const float l10 = lfc * 0.30102999566398120f;
        const float cc = -0.4f - 0.67f * l10, nn = 0.75f - 1.27f * l10;
        const float x = lpr * 0.30102999566398120f + cc;
        const float f1 = __fdividef(x, nn - 0.14f * x);
        fac += __fdividef(lfc, 1.0f + f1 * f1);                   // log2 F (Troe)
        out[u] = kf.w != 0.0f ? tc::ex2(fac) : s[u];
    }
}

// q_net of one reaction for one cell before any third-body / falloff factor (Eqs. 3-7),
// log2 domain: the contraction already holds sum nu' log2 C and sum nu'' log2 C - log2 K_c.
// Branch-free: kf.w zeroes the reverse rate of an irreversible reaction, and an empty slot's
// log2 k_f of -1e4 with S = 0 gives q = 0.
__device__ __forceinline__ float rate_plain(const CoefS *C, float sf, float sr, const CellF &c)
{
    const float4 kf = C->kf;
    const float lkf = fmaf(kf.z, c.invT, fmaf(kf.y, c.lg2T, kf.x));
    return fmaf(-kf.w, tc::ex2(sr + lkf), tc::ex2(sf + lkf));
}

// two values -> three packed BF16x2 words (hi, mid, lo terms; value a in the low halves)
__device__ __forceinline__ void split3x2(float a, float b, uint32_t &h, uint32_t &m, uint32_t &l)
{
    h = tc::pack_bf16x2(a, b);
    const float a1 = a - __uint_as_float(h << 16), b1 = b - __uint_as_float(h & 0xFFFF0000u);
    m = tc::pack_bf16x2(a1, b1);
    const float a2 = a1 - __uint_as_float(m << 16), b2 = b1 - __uint_as_float(m & 0xFFFF0000u);
    l = tc::pack_bf16x2(a2, b2);
}

// two values -> two packed BF16x2 words (hi, lo terms; value a in the low halves)
__device__ __forceinline__ void split2x2(float a, float b, uint32_t &h, uint32_t &l)
{
    h = tc::pack_bf16x2(a, b);
    l = tc::pack_bf16x2(a - __uint_as_float(h << 16), b - __uint_as_float(h & 0xFFFF0000u));
}

__device__ __forceinline__ void split3(float x, uint16_t &h, uint16_t &m, uint16_t &l)
{
    // x = hi + mid + lo with each term the nearest BF16 of the remaining residual
    const uint32_t ph = tc::pack_bf16x2(x, 0.0f) & 0xFFFFu;
    const float r1 = x - __uint_as_float(ph << 16);
    const uint32_t pm = tc::pack_bf16x2(r1, 0.0f) & 0xFFFFu;
    const float r2 = r1 - __uint_as_float(pm << 16);
    const uint32_t pl = tc::pack_bf16x2(r2, 0.0f) & 0xFFFFu;
    h = (uint16_t)ph;
    m = (uint16_t)pm;
    l = (uint16_t)pl;
}

template <int NSP, bool FOLD>
__global__ void __launch_bounds__(kThreads, 1) k_source_bf16(const Bf16Params p)
{
    using CL = Cols<NSP>;
    constexpr int SQ = NSP / 4;                   // species columns per warpgroup
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned base, offset on the shared array itself so that every access below
    // stays a shared-memory access (an integer round trip would make them generic)
    unsigned char *sm = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
    const uint32_t sbase = tc::smem_u32(sm);
    SmemTabs tabs;
    tabs.coef = (const CoefS *)(sm + p.o_coef);
    tabs.hmask = (const uint32_t *)(sm + p.o_hmask);
    tabs.fbase = (const int *)(tabs.hmask + NQ * p.nch);
    tabs.fq = (const FallQ *)(sm + p.o_fq);
    const GibbsS *gib = (const GibbsS *)(sm + p.o_gib);
    float *Ys = (float *)(sm + p.o_y);
    float *Ts = (float *)(sm + p.o_t);
    float *Ps = (float *)(sm + p.o_p);
    float *Ws = (float *)(sm + p.o_y);            // omega [128][ns], in the Y buffer between
                                                  // the next tile's prologue and its reload
    float *iW = (float *)(sm + p.o_iw);
    float *Psum = (float *)(sm + p.o_psum);      // [4][128] partial sums of z_k per warpgroup
    uint64_t *bars = (uint64_t *)(sm + p.o_bar);
    SmemCtl *ctl = (SmemCtl *)(bars + BAR_COUNT);
    auto BAR = [&](int i) { return tc::smem_u32(bars + i); };

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        const uint32_t cnt[BAR_COUNT] = {1, 1, 16, 16, 1, 16, 16, 1, 1, 16, 16, 1, 2, 16, 1};
        for (int i = 0; i < BAR_COUNT; ++i) tc::mbar_init(BAR(i), cnt[i]);
        tc::mbar_fence_init();
        ctl->abort = 0;
        ctl->mma1_issued = 0;
    }
    for (int k = tid; k < p.ns; k += kThreads) iW[k] = p.invW[k];
    if (warp == 1) {
        tc::tmem_alloc(tc::smem_u32(&ctl->tmem_base), kTmemCols);
        tc::tmem_relinquish();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = ctl->tmem_base;
    const int64_t n = p.n;

    if (warp == 0) {
        // ------------------------------------------------------------- tile loader
        if (lane == 0) {
            const uint32_t bt = p.blob_bytes;
            tc::mbar_arrive_expect_tx(BAR(BAR_BTAB), bt);
            for (uint32_t off = 0; off < bt; off += 16384)
                tc::bulk_g2s(sbase + off, (const unsigned char *)p.btab + off,
                             min(16384u, bt - off), BAR(BAR_BTAB));
            int it = 0;
            bool pending = false;
            for (int t = blockIdx.x; t < p.ntiles; t += gridDim.x, ++it) {
                if (!wait_bar(BAR(BAR_YEMPTY), (it & 1) ^ 1, ctl, p.status, 1)) break;
                const int64_t i0 = (int64_t)t * 128;
                if (p.stage_y && i0 + 128 <= n) {
                    const uint32_t yb = (uint32_t)(128 * p.ldY * 4);
                    tc::mbar_arrive_expect_tx(BAR(BAR_YFULL), yb + 1024);
                    tc::bulk_g2s(sbase + p.o_y, p.Y + i0 * p.ldY, yb, BAR(BAR_YFULL));
                    tc::bulk_g2s(sbase + p.o_t, p.T + i0, 512, BAR(BAR_YFULL));
                    tc::bulk_g2s(sbase + p.o_p, p.P + i0, 512, BAR(BAR_YFULL));
                    pending = true;
                } else {
                    tc::mbar_arrive(BAR(BAR_YFULL));
                    pending = false;
                }
            }
            // copies in flight are awaited before the CTA can exit
            if (pending) wait_bar(BAR(BAR_YFULL), (it - 1) & 1, ctl, p.status, 1);
            wait_bar(BAR(BAR_BTAB), 0, ctl, p.status, 1);
        }
    } else if (warp == 1 || warp == kMma2Warp) {
        // ------------------------------------------------------------- MMA issuers
        if (lane == 0) {
            constexpr uint32_t id1 = tc::idesc_bf16_f32(128, 2 * RC);
            constexpr uint32_t id2 = tc::idesc_bf16_f32(128, NSP);
            constexpr uint32_t id0 = tc::idesc_bf16_f32(128, kFacCols);
            const uint32_t b1 = sbase, b2 = sbase + p.o_b2, be = sbase + p.o_e;
            uint32_t u_d1 = 0, u_a2 = 0;        // contractions 1 and 2 issued so far
            bool ok = wait_bar(BAR(BAR_BTAB), 0, ctl, p.status, 2);
            constexpr uint32_t id1g = tc::idesc_bf16_f32(128, RC, true);
            auto issue_mma1 = [&](int c) {
                const uint32_t bc = b1 + (uint32_t)c * (2 * RC * NSP * 2);
#pragma unroll
                for (int s = 0; s < 3; ++s)
#pragma unroll
                    for (int kk = 0; kk < NSP / 16; ++kk)
                        tc::mma_ts(tmem + CL::D1, tmem + CL::A1 + s * (NSP / 2) + kk * 8,
                                   tc::sdesc_noswz(bc + kk * 256, 128, (NSP / 8) * 128), id1,
                                   (s | kk) != 0);
                // Gibbs layer into the reverse half: B = nu of contraction 2 ([species][reaction]
                // core matrices) read MN-major: K step = 2 species core rows, lbo = K stride
                const uint32_t bg = b2 + (uint32_t)c * (NSP * RC * 2);
#pragma unroll
                for (int s = 0; s < 3; ++s)
#pragma unroll
                    for (int kk = 0; kk < NSP / 16; ++kk)
                        tc::mma_ts(tmem + CL::D1 + RC, tmem + CL::AG + s * (NSP / 2) + kk * 8,
                                   tc::sdesc_noswz(bg + kk * 2 * (RC / 8) * 128, (RC / 8) * 128, 128),
                                   id1g, 1);
                tc::commit(BAR(BAR_D1FULL));
                ++u_d1;
            };
            // contraction 0: z (hi, lo) . (eff - 1) (hi, lo) as hi.hi + hi.lo + lo.hi into the
            // multiplier columns.  Issued after chunk 0's contraction 1 (it then runs while
            // chunk 0's S is read out) unless chunk 0 reads multipliers; either way a D1FULL
            // commit of this thread covers it before the first chunk that reads them, and its
            // operand columns are free for chunk 0's q_net at ZFREE.
            auto issue_mma0 = [&]() {
#pragma unroll
                for (int s = 0; s < 3; ++s)
#pragma unroll
                    for (int kk = 0; kk < NSP / 16; ++kk)
                        tc::mma_ts(tmem + CL::FC, tmem + CL::A2 + (s == 2 ? NSP / 2 : 0) + kk * 8,
                                   tc::sdesc_noswz(be + (s == 1 ? kFacCols * NSP * 2 : 0) + kk * 256,
                                                   128, (NSP / 8) * 128),
                                   id0, (s | kk) != 0);
                tc::commit(BAR(BAR_ZFREE));
            };
            auto mma2 = [&](int c) {
                const uint32_t bc = b2 + (uint32_t)c * (NSP * RC * 2);
#pragma unroll
                for (int s = 0; s < 2; ++s)
#pragma unroll
                    for (int kk = 0; kk < RC / 16; ++kk)
                        tc::mma_ts(tmem + CL::D2, tmem + CL::A2 + s * (RC / 2) + kk * 8,
                                   tc::sdesc_noswz(bc + kk * 256, 128, (RC / 8) * 128), id2,
                                   (c | s | kk) != 0);
                tc::commit(BAR(BAR_A2EMPTY));
                ++u_a2;
                if (c == p.nch - 1) tc::commit(BAR(BAR_D2FULL));
            };
            int it = 0;
            if (warp == 1) {
                for (int t = blockIdx.x; ok && t < p.ntiles; t += gridDim.x, ++it) {
                    if (!(ok = wait_bar(BAR(BAR_A1FULL), it & 1, ctl, p.status, 2))) break;
                    tc::fence_after();
                    // chunk 0 reads multipliers: contraction 0 first (its D1FULL covers it)
                    if (p.fac_chunk0) issue_mma0();
                    // contraction 1 of each chunk as soon as the previous S has been read out
                    for (int c = 0; ok && c < p.nch; ++c) {
                        if (!(ok = wait_bar(BAR(BAR_D1EMPTY), (u_d1 & 1) ^ 1, ctl, p.status, 2)))
                            break;
                        tc::fence_after();
                        issue_mma1(c);
                        ctl->mma1_issued = (int)u_d1;
                        if (c == 0 && !p.fac_chunk0) issue_mma0();
                    }
                    // completes when every contraction 1 of the tile has read its operands
                    if (ok) tc::commit(BAR(BAR_A1FREE));
                }
            } else {
                // contraction 2 in chunk order (the omega accumulation order, hence the
                // rounding, is fixed), the first of a tile once omega of the tile before has
                // been read out
                for (int t = blockIdx.x; ok && t < p.ntiles; t += gridDim.x, ++it) {
                    if (!(ok = wait_bar(BAR(BAR_D2EMPTY), (it & 1) ^ 1, ctl, p.status, 2))) break;
                    for (int c = 0; ok && c < p.nch; ++c) {
                        if (!(ok = wait_bar(BAR(BAR_A2FULL), u_a2 & 1, ctl, p.status, 2))) break;
                        // Let contraction 1 of the next chunk go first: it gates the epilogue,
                        // while this one fills the pipe during the next S read-out.  Only the
                        // order on the tensor pipe depends on this (the two are independent),
                        // so the wait is short and bounded and then proceeds regardless.
                        if (c + 1 < p.nch)
                            for (int spin = 0; spin < 4096 && ctl->mma1_issued < (int)u_a2 + 2; ++spin)
                                __nanosleep(20);
                        tc::fence_after();
                        mma2(c);
                    }
                }
            }
            // every MMA issued (by both issuers) has completed before tensor memory is released
            tc::commit(BAR(BAR_DRAIN));
            wait_bar(BAR(BAR_DRAIN), 0, ctl, p.status, 2);
        }
    } else if (warp < kMma2Warp) {
        // ------------------------------------------------------------- epilogue
        const int ew = warp - kEpiWarp0;             // 0..15
        const int g = ew >> 2;                        // warpgroup 0..3: quarter of each chunk
        const int q = warp & 3;                       // lane quarter of tensor memory
        const int row = q * 32 + lane;
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        const int ns = p.ns;
        int it = 0, u = 0;
        bool ok = wait_bar(BAR(BAR_BTAB), 0, ctl, p.status, 3);   // coefficients in smem
        CellF cf;
        // ---- prologue of tile t: features, X and split log2 X (Eq. 4 input layer); ends
        // with the tile's contraction-1 operands in tensor memory (A1FULL)
        auto prologue = [&](int t, int itp) -> bool {
            const int64_t i0 = (int64_t)t * 128;
            const int64_t ci = i0 + row;
            const bool full = p.stage_y && i0 + 128 <= n;
            if (!wait_bar(BAR(BAR_YFULL), itp & 1, ctl, p.status, 3)) return false;
            // ---- prologue: features, X and split log2 X (Eq. 4 input layer)
            float Tc = 1000.0f, Pc = 1.0e6f;
            const float *yrow = nullptr;
            if (full) {
                Tc = Ts[row];
                Pc = Ps[row];
                yrow = Ys + (int64_t)row * p.ldY;
            } else if (ci < n) {
                Tc = __ldg(p.T + ci);
                Pc = __ldg(p.P + ci);
                yrow = p.Y + ci * p.ldY;
            }
            cf.lg2T = log2f(Tc);
            cf.invT = 1.0f / Tc;
            cf.tau = Tc * 1e-3f;
            cf.tau2 = cf.tau * cf.tau;
            cf.rg = Tc >= p.t_mid ? 1 : 0;
            cf.lgct = log2f(Pc) - p.lg2R - cf.lg2T;
            // This warpgroup's quarter of the species columns: z_k = Y_k / W_k, whose log2
            // goes to the contraction; X_k = z_k / sum_k z_k is completed by the column
            // ns + 1 below (log2 c_tot - log2 sum, weighted by the reaction order).
            float psum = 0.0f;
            uint32_t wh[SQ / 2], wm[SQ / 2], wl[SQ / 2];   // log2 z, three BF16 terms
            uint32_t gh[SQ / 2], gm[SQ / 2], gl[SQ / 2];   // G, three BF16 terms
            uint32_t zh[SQ / 2], zl[SQ / 2];               // z, two BF16 terms (contraction 0)
#pragma unroll
            for (int e = 0; e < SQ / 2; ++e) {
                float lx[2], gk[2], zz[2];
#pragma unroll
                for (int hlf = 0; hlf < 2; ++hlf) {
                    const int k = g * SQ + 2 * e + hlf;
                    lx[hlf] = 0.0f;
                    gk[hlf] = 0.0f;
                    zz[hlf] = 0.0f;
                    if (k < ns) {
                        const float z = yrow ? fmaxf(yrow[k], 0.0f) * iW[k] : 0.0f;
                        psum += z;
                        zz[hlf] = z;
                        lx[hlf] = fmaxf(tc::lg2(z), kLog2Floor);
                        // Gibbs layer (Eq. 10) for this species at this cell's temperature
                        const float4 g0 = *(const float4 *)&gib[k].c[cf.rg][0];
                        const float4 g1 = *(const float4 *)&gib[k].c[cf.rg][4];
                        const float pt = fmaf(fmaf(fmaf(g1.y, cf.tau, g1.x), cf.tau, g0.w), cf.tau, g0.z);
                        gk[hlf] = fmaf(pt, cf.tau, fmaf(g1.z, cf.invT, fmaf(g0.y, cf.lg2T, g0.x)));
                    } else if (k == ns) {
                        lx[hlf] = cf.lgct;            // third-body c_tot column
                    } else if (FOLD && k >= ns + 2 && k < ns + 2 + kFoldRows) {
                        // Arrhenius features 1, log2 T, 1/T, each against three rows
                        const int f = (k - ns - 2) / 3;
                        lx[hlf] = f == 0 ? 1.0f : (f == 1 ? cf.lg2T : cf.invT);
                    }
                }
                split3x2(lx[0], lx[1], wh[e], wm[e], wl[e]);
                split3x2(gk[0], gk[1], gh[e], gm[e], gl[e]);
                split2x2(zz[0], zz[1], zh[e], zl[e]);
            }
            // the previous tile's contractions 1 have read their operands
            if (itp > 0 && !wait_bar(BAR(BAR_A1FREE), (itp - 1) & 1, ctl, p.status, 3)) return false;
            // ... and the previous tile's last contraction 2 has read its q_net operand, whose
            // columns take z now
            if (!wait_bar(BAR(BAR_A2EMPTY), (u & 1) ^ 1, ctl, p.status, 3)) return false;
            tc::fence_after();
            const uint32_t az = tmem + lane_off + CL::A2 + g * (SQ / 2);
            const uint32_t a1 = tmem + lane_off + CL::A1 + g * (SQ / 2);
            const uint32_t ag = tmem + lane_off + CL::AG + g * (SQ / 2);
            if constexpr (SQ / 2 == 8) {
                tc::tmem_st8(a1 + 0 * (NSP / 2), wh);
                tc::tmem_st8(a1 + 1 * (NSP / 2), wm);
                tc::tmem_st8(a1 + 2 * (NSP / 2), wl);
                tc::tmem_st8(ag + 0 * (NSP / 2), gh);
                tc::tmem_st8(ag + 1 * (NSP / 2), gm);
                tc::tmem_st8(ag + 2 * (NSP / 2), gl);
                tc::tmem_st8(az, zh);
                tc::tmem_st8(az + NSP / 2, zl);
            } else {
                static_assert(SQ / 2 == 4, "warpgroup species quarter of 8 or 16 columns");
                tc::tmem_st4(a1 + 0 * (NSP / 2), wh);
                tc::tmem_st4(a1 + 1 * (NSP / 2), wm);
                tc::tmem_st4(a1 + 2 * (NSP / 2), wl);
                tc::tmem_st4(ag + 0 * (NSP / 2), gh);
                tc::tmem_st4(ag + 1 * (NSP / 2), gm);
                tc::tmem_st4(ag + 2 * (NSP / 2), gl);
                tc::tmem_st4(az, zh);
                tc::tmem_st4(az + NSP / 2, zl);
            }
            tc::tmem_wait_st();
            Psum[g * 128 + row] = psum;
            __syncwarp();
            if (lane == 0) {
                // the first tile's Y buffer is free now; later ones hold omega of the tile
                // before until it has been stored
                if (itp == 0) tc::mbar_arrive(BAR(BAR_YEMPTY));
                tc::mbar_arrive(BAR(BAR_XREADY));
            }
            if (!wait_bar(BAR(BAR_XREADY), itp & 1, ctl, p.status, 3)) return false;
            {
                const float sum = Psum[row] + Psum[128 + row] + Psum[256 + row] + Psum[384 + row];
                cf.inv_sum = sum > 0.0f ? 1.0f / sum : 0.0f;
                const int kn = ns + 1;                    // normalisation column
                if (kn / SQ == g) {
                    // the packed word holding column kn; its other half is column kn - 1
                    // (= ns, log2 c_tot) or kn + 1 (the first Arrhenius feature, 1, or
                    // padding, zero)
                    const float other = (kn & 1) ? cf.lgct : (FOLD ? 1.0f : 0.0f);
                    const float vn = sum > 0.0f ? cf.lgct - log2f(sum) : 0.0f;
                    uint16_t ho, mo, lo_, hn, mn, ln;
                    split3(other, ho, mo, lo_);
                    split3(vn, hn, mn, ln);
                    auto pk = [&](uint16_t o, uint16_t nn) {
                        return (kn & 1) ? ((uint32_t)o | ((uint32_t)nn << 16))
                                        : ((uint32_t)nn | ((uint32_t)o << 16));
                    };
                    const uint32_t col = tmem + lane_off + CL::A1 + kn / 2;
                    tc::tmem_st1(col + 0 * (NSP / 2), pk(ho, hn));
                    tc::tmem_st1(col + 1 * (NSP / 2), pk(mo, mn));
                    tc::tmem_st1(col + 2 * (NSP / 2), pk(lo_, ln));
                }
                tc::tmem_wait_st();
                tc::fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(BAR(BAR_A1FULL));
            }
            return true;
        };
        if ((int)blockIdx.x < p.ntiles) ok = ok && prologue(blockIdx.x, 0);
        for (int t = blockIdx.x; ok && t < p.ntiles; t += gridDim.x, ++it) {
            const int64_t i0 = (int64_t)t * 128;
            const int64_t ci = i0 + row;
            // ---- every chunk, this warpgroup's quarter of its reactions
            for (int c = 0; c < p.nch; ++c, ++u) {
                if (!(ok = wait_bar(BAR(BAR_D1FULL), u & 1, ctl, p.status, 3))) break;
                tc::fence_after();
                uint32_t sf[RH], sr[RH], fv[8];
                const uint32_t d1 = tmem + lane_off + CL::D1 + g * RH;
                // both halves of contraction 1 and this quarter's (at most 8) multipliers,
                // consecutive columns, behind one completion wait
                const int mq = c * NQ + g;
                const uint32_t hm = tabs.hmask[mq];
                const int lb = hm ? tabs.fbase[mq] : 0;
                tc::tmem_ld16_nw(d1, sf);
                tc::tmem_ld16_nw(d1 + RC, sr);
                if (hm) {
                    tc::tmem_ld8_nw(tmem + lane_off + CL::FC + lb, fv);
                } else {
#pragma unroll
                    for (int e = 0; e < 8; ++e) fv[e] = 0u;
                }
                tc::tmem_wait_ld_tie(sf, sr, fv);
                tc::fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(BAR(BAR_D1EMPTY));
                const int j0 = c * RC + g * RH;
                float q[RH];
                if constexpr (FOLD) {
#pragma unroll
                    for (int r = 0; r < RH; ++r)
                        q[r] = tc::ex2(__uint_as_float(sf[r])) - tc::ex2(__uint_as_float(sr[r]));
                } else {
#pragma unroll
                    for (int r = 0; r < RH; ++r)
                        q[r] = rate_plain(tabs.coef + j0 + r, __uint_as_float(sf[r]),
                                          __uint_as_float(sr[r]), cf);
                }
                if (hm) {
                    // the quarter's third-body / falloff reactions sit in its first 8 slots
                    // (falloff in 0..3); their columns hold sum_k (eff_k - 1) z_k (0 for the
                    // other slots), so M / c_tot = 1 + that / sum_k z_k
                    float s8[8], fo[4];
#pragma unroll
                    for (int r = 0; r < 8; ++r)
                        s8[r] = fmaf(__uint_as_float(fv[r]), cf.inv_sum, 1.0f);
                    falloff4(tabs.fq + 4 * (lb / 8), s8, cf, fo);
#pragma unroll
                    for (int r = 0; r < 4; ++r) q[r] *= fo[r];
#pragma unroll
                    for (int r = 4; r < 8; ++r) q[r] *= s8[r];
                }
                uint32_t hw[RH / 2], lw[RH / 2];
#pragma unroll
                for (int r = 0; r < RH; r += 2) {
                    const uint32_t h = tc::pack_bf16x2(q[r], q[r + 1]);
                    const float r0 = q[r] - __uint_as_float(h << 16);
                    const float r1 = q[r + 1] - __uint_as_float(h & 0xFFFF0000u);
                    hw[r / 2] = h;
                    lw[r / 2] = tc::pack_bf16x2(r0, r1);
                }
                if (!(ok = wait_bar(BAR(BAR_A2EMPTY), (u & 1) ^ 1, ctl, p.status, 3))) break;
                // chunk 0: contraction 0 has read z from these columns
                if (c == 0 && !(ok = wait_bar(BAR(BAR_ZFREE), it & 1, ctl, p.status, 3))) break;
                tc::fence_after();
                const uint32_t a2 = tmem + lane_off + CL::A2 + g * (RH / 2);
                tc::tmem_st8(a2, hw);
                tc::tmem_st8(a2 + RC / 2, lw);
                tc::tmem_wait_st();
                tc::fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(BAR(BAR_A2FULL));
            }
            if (!ok) break;
            // ---- the next tile's prologue first: it needs none of this tile's tensor memory
            // (every contraction 1 of this tile has completed), so its contraction 1 can
            // start while this tile's omega is read out
            const int t_next = t + gridDim.x;
            if (t_next < p.ntiles && !(ok = prologue(t_next, it + 1))) break;
            // ---- omega of the tile: tensor memory -> shared (the Y buffer, read by the next
            // tile's prologue already) -> one coalesced bulk store; then the buffer is free
            // for the tile after next (YEMPTY)
            if (!(ok = wait_bar(BAR(BAR_D2FULL), it & 1, ctl, p.status, 3))) break;
            tc::fence_after();
            {
                uint32_t w[SQ];
                const uint32_t d2 = tmem + lane_off + CL::D2 + g * SQ;
                if constexpr (SQ == 16) tc::tmem_ld16(d2, w);
                else tc::tmem_ld8(d2, w);
                tc::fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(BAR(BAR_D2EMPTY));
                if (p.stage_y) {
#pragma unroll
                    for (int e = 0; e < SQ; ++e) {
                        const int k = g * SQ + e;
                        if (k < ns) Ws[row * ns + k] = __uint_as_float(w[e]);
                    }
                } else if (ci < n) {                  // no staging buffer: direct stores
                    float *orow = p.om + ci * p.ldO;
#pragma unroll
                    for (int e = 0; e < SQ; ++e) {
                        const int k = g * SQ + e;
                        if (k < ns) orow[k] = __uint_as_float(w[e]);
                    }
                }
            }
            if (p.stage_y) {
                tc::fence_proxy_async_smem();            // visible to the bulk store
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(BAR(BAR_WREADY));
                if (!(ok = wait_bar(BAR(BAR_WREADY), it & 1, ctl, p.status, 3))) break;
                if (p.bulk_out && i0 + 128 <= n) {
                    if (ew == 0 && lane == 0) {
                        tc::bulk_s2g(p.om + i0 * p.ldO, sbase + p.o_y, (uint32_t)(128 * ns * 4));
                        tc::bulk_commit();
                        tc::bulk_wait_read0();
                    }
                } else {
                    for (int r = ew; r < 128; r += kEpiWarps) {
                        const int64_t i = i0 + r;
                        if (i >= n) break;
                        float *orow = p.om + i * p.ldO;
                        for (int k = lane; k < ns; k += 32) orow[k] = Ws[r * ns + k];
                    }
                }
            }
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(BAR(BAR_YEMPTY));
        }
    }
    if (warp == kEpiWarp0 && lane == 0) tc::bulk_wait0();   // omega stores have landed
    tc::fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc::fence_after();
        tc::tmem_dealloc(tmem, kTmemCols);
    }
}

// ---------------------------------------------------------------------------------------
// host side: tables, launch
// ---------------------------------------------------------------------------------------

static uint16_t bf16_of_int(int v)
{
    float f = (float)v;
    uint32_t u;
    memcpy(&u, &f, 4);
    return (uint16_t)(u >> 16);              // exact for |v| <= 256
}

static uint16_t bf16_rn(float f)
{
    uint32_t u;
    memcpy(&u, &f, 4);
    return (uint16_t)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);   // nearest, ties to even
}

static double f_of_bf16(uint16_t h)
{
    const uint32_t u = (uint32_t)h << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

// x = hi + mid + lo, each term the nearest BF16 of the remaining residual
static void bf16_split3(double x, uint16_t (&t)[3])
{
    for (int i = 0; i < 3; ++i) {
        t[i] = bf16_rn((float)x);
        x -= f_of_bf16(t[i]);
    }
}

chem_status bf16_build_tables(chem_mech *m, const chem_mech_desc *d)
{
    const int ns = d->n_species, nr = d->n_reactions;
    // columns: species 0..ns-1, then log2 c_tot (third-body factor) and the
    // normalisation column log2 c_tot - log2 sum_k z_k (weighted by the reaction order)
    int nsp = ((ns + 2 + 15) / 16) * 16;
    if (nsp <= 32) nsp = 32;
    else if (nsp <= 64) nsp = 64;
    else return set_error(CHEM_EUNSUPPORTED, "split-BF16 path supports up to 62 species");
    const int nch = (nr + RC - 1) / RC;
    const int nrp = nch * RC;
    // the Arrhenius layer rides in contraction 1 when nine padding rows are free
    const bool fold = ns + 2 + kFoldRows <= nsp;
    const int kf0 = ns + 2;
    // Reactions without a third-body or falloff factor fill the first chunks (spread evenly
    // over their slots); those with one go to the first 8 slots of the last K chunks'
    // quarters (falloff ones round-robin into slots 0..3, third-body ones into the least
    // filled quarter), with the rest of the plain reactions.  Each such quarter owns 8
    // multiplier columns: contraction 0 fills them with its third-body sums.
    std::vector<int> plain, fall, tbr;
    for (int j = 0; j < nr; ++j)
        (d->kind[j] == 0 ? plain : d->kind[j] == CHEM_RXN_THIRD_BODY ? tbr : fall).push_back(j);
    const int S = (int)(fall.size() + tbr.size());
    int K = 0;
    if (S) K = std::max((S + NQ * 8 - 1) / (NQ * 8), ((int)fall.size() + NQ * 4 - 1) / (NQ * 4));
    if (K > nch || NQ * K * 8 > kFacCols)
        return set_error(CHEM_EUNSUPPORTED,
                         "split-BF16 path: %d third-body / falloff reactions (%d falloff) exceed "
                         "its %d multiplier columns", S, (int)fall.size(), kFacCols);
    std::vector<int> order(nrp, -1);        // slot -> reaction (-1: padding)
    size_t pi = 0;
    {
        const int head_slots = (nch - K) * RC;
        const int n_head = std::min((int)plain.size(), head_slots);
        for (int i = 0; i < n_head; ++i)
            order[(size_t)((int64_t)i * head_slots / n_head)] = plain[pi++];
        const int nqt = NQ * K;
        std::vector<int> fill(nqt, 0);
        for (size_t i = 0; i < fall.size(); ++i) {
            const int qq = (int)(i % nqt);
            order[(size_t)((nch - K) * NQ + qq) * RH + fill[qq]++] = fall[i];
        }
        for (size_t i = 0; i < tbr.size(); ++i) {
            int qq = 0;
            for (int x = 1; x < nqt; ++x)
                if (fill[x] < fill[qq]) qq = x;
            order[(size_t)((nch - K) * NQ + qq) * RH + fill[qq]++] = tbr[i];
        }
        for (int jj = head_slots; jj < nrp && pi < plain.size(); ++jj)
            if (order[jj] < 0) order[jj] = plain[pi++];
    }
    if (pi != plain.size()) return set_error(CHEM_EUNSUPPORTED, "split-BF16 path: slot layout");
    std::vector<uint16_t> b1((size_t)nch * 2 * RC * nsp, 0), b2((size_t)nch * nsp * RC, 0);
    const size_t e_term = (size_t)kFacCols * nsp;
    std::vector<uint16_t> eb(2 * e_term, 0);          // eff - 1: [term][column][species]
    std::vector<CoefS> cf(nrp);
    // per chunk quarter: holds third-body / falloff reactions; its first multiplier column
    std::vector<uint32_t> hmask((size_t)nch * 2 * NQ, 0);
    std::vector<int> qrank((size_t)nch * NQ, -1);
    int nq_special = 0;
    for (int jj = 0; jj < nrp; ++jj)
        if (order[jj] >= 0 && d->kind[order[jj]] != 0 && qrank[jj / RH] < 0) {
            qrank[jj / RH] = nq_special++;
            hmask[jj / RH] = 1;
            hmask[(size_t)nch * NQ + jj / RH] = (uint32_t)(8 * qrank[jj / RH]);
        }
    FallQ neutral;
    memset(&neutral, 0, sizeof neutral);
    neutral.troe = make_float4(1.0f, 0.0f, 0.0f, 0.0f);
    neutral.t2 = make_float4(1e30f, 0.0f, 0.0f, 0.0f);
    std::vector<FallQ> fq((size_t)std::max(nq_special, 1) * 4, neutral);
    auto b1_at = [&](int c, int r, int k) -> uint16_t & {
        return b1[(size_t)c * 2 * RC * nsp + ((r / 8) * (nsp / 8) + k / 8) * 64 + (r % 8) * 8 + k % 8];
    };
    auto b2_at = [&](int c, int nrow, int r) -> uint16_t & {
        return b2[(size_t)c * nsp * RC + ((nrow / 8) * (RC / 8) + r / 8) * 64 + (nrow % 8) * 8 + r % 8];
    };
    auto e_at = [&](int term, int n, int k) -> uint16_t & {
        return eb[term * e_term + ((n / 8) * (nsp / 8) + k / 8) * 64 + (n % 8) * 8 + k % 8];
    };
    for (int jj = 0; jj < nrp; ++jj) {
        CoefS &C = cf[jj];
        memset(&C, 0, sizeof C);
        const int c = jj / RC, r = jj % RC;
        if (order[jj] < 0) {                    // padding slot: q = 0
            C.kf = make_float4(kDead, 0, 0, 0);
            if (fold) {
                uint16_t t3[3];
                bf16_split3(kDead, t3);
                for (int i = 0; i < 3; ++i) b1_at(c, r, kf0 + i) = b1_at(c, RC + r, kf0 + i) = t3[i];
            }
            continue;
        }
        const int j = order[jj];
        const int kind = d->kind[j];
        const double *ar = d->arrh + (size_t)j * 3;
        int ordf = 0, ordr = 0;
        for (int k = 0; k < ns; ++k) {
            const int f = d->nu_f[(size_t)j * ns + k], pr = d->nu_r[(size_t)j * ns + k];
            ordf += f;
            ordr += pr;
            b1_at(c, r, k) = bf16_of_int(f);
            b1_at(c, RC + r, k) = bf16_of_int(pr);
            b2_at(c, k, r) = bf16_of_int(pr - f);
        }
        const int tbx = kind == CHEM_RXN_THIRD_BODY ? 1 : 0;   // log2 M = log2 c_tot + log2(M/c_tot)
        b1_at(c, r, ns) = bf16_of_int(tbx);
        b1_at(c, RC + r, ns) = bf16_of_int(tbx);
        b1_at(c, r, ns + 1) = bf16_of_int(ordf);
        b1_at(c, RC + r, ns + 1) = bf16_of_int(ordr);
        C.kf = make_float4((float)(ar[0] * kLog2e), (float)ar[1], (float)(-ar[2] * kLog2e),
                           d->reversible[j] ? 1.0f : 0.0f);
        if (fold) {
            // rows kf0 + 3 f + i: term i of the coefficient of feature f (1, log2 T, 1/T)
            const double co[3] = {ar[0] * kLog2e, ar[1], -ar[2] * kLog2e};
            for (int f = 0; f < 3; ++f) {
                uint16_t t3[3];
                bf16_split3(co[f], t3);
                for (int i = 0; i < 3; ++i) {
                    b1_at(c, r, kf0 + 3 * f + i) = t3[i];
                    if (d->reversible[j]) b1_at(c, RC + r, kf0 + 3 * f + i) = t3[i];
                }
            }
            if (!d->reversible[j]) {
                uint16_t t3[3];
                bf16_split3(kDead, t3);
                for (int i = 0; i < 3; ++i) b1_at(c, RC + r, kf0 + i) = t3[i];
            }
        }
        if (kind == 0) continue;
        // third-body sum column (contraction 0): eff - 1 in two BF16 terms
        const int pos = jj % RH, col = 8 * qrank[jj / RH] + pos;
        if (pos >= 8 || (kind != CHEM_RXN_THIRD_BODY && pos >= 4))
            return set_error(CHEM_EUNSUPPORTED, "split-BF16 path: multiplier slot layout");
        for (int k = 0; k < ns; ++k) {
            const double e = (d->eff ? d->eff[(size_t)j * ns + k] : 1.0) - 1.0;
            const uint16_t hi = bf16_rn((float)e);
            e_at(0, col, k) = hi;
            e_at(1, col, k) = bf16_rn((float)(e - f_of_bf16(hi)));
        }
        if (kind != CHEM_RXN_THIRD_BODY) {
            FallQ &F = fq[(size_t)4 * qrank[jj / RH] + pos];
            const double *al = d->arrh_low + (size_t)j * 3;
            F.kf = make_float4(C.kf.x, C.kf.y, C.kf.z, 1.0f);
            F.k0 = make_float4((float)(al[0] * kLog2e), (float)al[1], (float)(-al[2] * kLog2e), 0.f);
            if (kind == CHEM_RXN_TROE) {
                const double *tp = d->troe + (size_t)j * 4;
                F.troe = make_float4((float)(1.0 - tp[0]), (float)tp[0], (float)(kLog2e / tp[1]),
                                     (float)(kLog2e / tp[2]));
                if (tp[3] > 0.0) F.t2 = make_float4((float)(tp[3] * kLog2e), 0, 0, 0);
            }
        }
    }
    // Gibbs layer per species (log2 units, the standard concentration folded into the bias):
    // G = (a1 - a7) log2e - log2(p_ref/R) + (1 - a1) log2 T - a2/2 T log2e - a3/6 T^2 log2e
    //     - a4/12 T^3 log2e - a5/20 T^4 log2e + a6 log2e / T
    std::vector<GibbsS> gb(ns);
    const double lg2_pref_R = log2(d->p_ref / kR);
    for (int k = 0; k < ns; ++k) {
        memset(&gb[k], 0, sizeof gb[k]);
        for (int rg = 0; rg < 2; ++rg) {
            const double *a = d->nasa7 + (size_t)k * 14 + (size_t)rg * 7;
            const double cc[7] = {(a[0] - a[6]) * kLog2e - lg2_pref_R, 1.0 - a[0],
                                  -a[1] / 2.0 * 1e3 * kLog2e, -a[2] / 6.0 * 1e6 * kLog2e,
                                  -a[3] / 12.0 * 1e9 * kLog2e, -a[4] / 20.0 * 1e12 * kLog2e,
                                  a[5] * kLog2e};
            for (int q = 0; q < 7; ++q) gb[k].c[rg][q] = (float)cc[q];
        }
    }
    std::vector<float> invW(ns);
    for (int k = 0; k < ns; ++k) invW[k] = (float)(1.0 / d->mol_weight[k]);

    // B1 | B2 | E | coefficients | quarter masks | falloff | Gibbs: contiguous, copied to
    // shared memory by one bulk transfer (16-byte granules)
    auto a16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
    auto a256 = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t ob1 = 0, ob2 = b1.size() * 2, oe = ob2 + b2.size() * 2, ocf = oe + eb.size() * 2;
    const size_t ohm = a16(ocf + cf.size() * sizeof(CoefS));
    const size_t ofq = a16(ohm + hmask.size() * 4);
    const size_t ogb = a16(ofq + fq.size() * sizeof(FallQ));
    const size_t blob = a16(ogb + gb.size() * sizeof(GibbsS));
    const size_t oiw = a256(blob), ost = a256(oiw + invW.size() * 4), total = a256(ost + 16);
    std::vector<unsigned char> h(total, 0);
    memcpy(h.data() + ob1, b1.data(), b1.size() * 2);
    memcpy(h.data() + ob2, b2.data(), b2.size() * 2);
    memcpy(h.data() + oe, eb.data(), eb.size() * 2);
    memcpy(h.data() + ocf, cf.data(), cf.size() * sizeof(CoefS));
    memcpy(h.data() + ohm, hmask.data(), hmask.size() * 4);
    memcpy(h.data() + ofq, fq.data(), fq.size() * sizeof(FallQ));
    memcpy(h.data() + ogb, gb.data(), gb.size() * sizeof(GibbsS));
    memcpy(h.data() + oiw, invW.data(), invW.size() * 4);
    Bf16Tables *t = new (std::nothrow) Bf16Tables();
    if (!t) return set_error(CHEM_ENOMEM, "host allocation failed");
    cudaError_t e = cudaMalloc(&t->d_blob, total);
    if (e != cudaSuccess) {
        delete t;
        return set_error(CHEM_ENOMEM, "cudaMalloc: %s", cudaGetErrorString(e));
    }
    e = cudaMemcpy(t->d_blob, h.data(), total, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(t->d_blob);
        delete t;
        return set_error(CHEM_ECUDA, "cudaMemcpy: %s", cudaGetErrorString(e));
    }
    unsigned char *base = (unsigned char *)t->d_blob;
    t->nsp = nsp;
    t->fold = fold;
    t->fac_chunk0 = 0;
    for (int q = 0; q < NQ; ++q) t->fac_chunk0 |= hmask[q] ? 1 : 0;
    t->nch = nch;
    t->b1_bytes = b1.size() * 2;
    t->blob_bytes = blob;
    t->o_b2 = (uint32_t)ob2;
    t->o_e = (uint32_t)oe;
    t->o_coef = (uint32_t)ocf;
    t->o_hmask = (uint32_t)ohm;
    t->o_fq = (uint32_t)ofq;
    t->o_gib = (uint32_t)ogb;
    t->btab = (const uint16_t *)(base + ob1);
    t->invW = (const float *)(base + oiw);
    t->status = (int *)(base + ost);
    m->bf16 = t;
    m->have_bf16 = true;
    m->device_bytes += total;
    return CHEM_OK;
}

void bf16_free_tables(void *p)
{
    Bf16Tables *t = (Bf16Tables *)p;
    if (!t) return;
    cudaFree(t->d_blob);
    delete t;
}

int *bf16_status_word(const chem_mech *m)
{
    return m->have_bf16 ? ((Bf16Tables *)m->bf16)->status : nullptr;
}

static int sm_count(int dev)
{
    static int cache[64] = {0};
    if (dev < 0 || dev >= 64) return 148;
    if (!cache[dev]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cache[dev] = v > 0 ? v : 148;
    }
    return cache[dev];
}

template <int NSP, bool FOLD>
static chem_status launch_nsp(const Bf16Params &prm, size_t smem, cudaStream_t s, int dev)
{
    static std::atomic<uint32_t> done{0};
    const uint32_t bit = 1u << (dev & 31);
    if (!(done.load() & bit)) {
        cudaError_t e = cudaFuncSetAttribute(k_source_bf16<NSP, FOLD>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             227 * 1024);
        if (e != cudaSuccess)
            return set_error(CHEM_ECUDA, "split-BF16 attribute: %s", cudaGetErrorString(e));
        done.fetch_or(bit);
    }
    const int grid = std::min(prm.ntiles, sm_count(dev));
    k_source_bf16<NSP, FOLD><<<grid, kThreads, smem, s>>>(prm);
    g_launches.fetch_add(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(CHEM_ECUDA, "split-BF16 launch: %s", cudaGetErrorString(e));
    return CHEM_OK;
}

chem_status launch_source_bf16(const chem_mech *m, int64_t n, const float *T, const float *P,
                               const float *Y, int64_t ldY, float *om, int64_t ldO,
                               cudaStream_t s)
{
    if (!m->have_bf16)
        return set_error(CHEM_EUNSUPPORTED, "split-BF16 path not available for this mechanism");
    const Bf16Tables *t = (const Bf16Tables *)m->bf16;
    Bf16Params prm;
    memset(&prm, 0, sizeof prm);
    prm.T = T;
    prm.P = P;
    prm.Y = Y;
    prm.om = om;
    prm.n = n;
    prm.ldY = ldY;
    prm.ldO = ldO;
    prm.ns = m->ns;
    prm.nch = t->nch;
    prm.fac_chunk0 = t->fac_chunk0;
    prm.bulk_out = (ldO == m->ns && (uintptr_t)om % 16 == 0) ? 1 : 0;
    prm.ntiles = (int)((n + 127) / 128);
    prm.btab = t->btab;
    prm.blob_bytes = (uint32_t)t->blob_bytes;
    prm.invW = t->invW;
    prm.t_mid = (float)m->t_mid;
    prm.lg2R = (float)log2(kR);
    prm.status = t->status;
    if ((int64_t)((n + 127) / 128) > 0x7fffffff) return set_error(CHEM_EINVAL, "n_cells too large");
    // shared memory layout
    auto al = [](size_t x, size_t a) { return (x + a - 1) & ~(a - 1); };
    prm.o_b2 = t->o_b2;
    prm.o_e = t->o_e;
    prm.o_coef = t->o_coef;
    prm.o_hmask = t->o_hmask;
    prm.o_fq = t->o_fq;
    prm.o_gib = t->o_gib;
    size_t off = al(prm.blob_bytes, 128);
    const size_t ybytes = (size_t)128 * ldY * 4;
    const size_t fixed = 2 * 512 + al(m->ns * 4, 128) + 2048 + BAR_COUNT * 8 + 64 + 1024;
    const bool aligned = ((uintptr_t)Y % 16 == 0) && ((uintptr_t)T % 16 == 0) && ((uintptr_t)P % 16 == 0);
    prm.stage_y = aligned && (off + ybytes + fixed <= 227 * 1024) ? 1 : 0;
    prm.o_y = (uint32_t)off;
    if (prm.stage_y) off = al(off + ybytes, 128);
    prm.o_t = (uint32_t)off;
    off += 512;
    prm.o_p = (uint32_t)off;
    off += 512;
    prm.o_iw = (uint32_t)off;
    off = al(off + m->ns * 4, 128);
    prm.o_psum = (uint32_t)off;
    off += 4 * 128 * 4;
    prm.o_bar = (uint32_t)off;
    off += BAR_COUNT * 8 + 64;
    const size_t smem = off + 1024;          // room to align the base to 1024 bytes
    if (smem > 227 * 1024)
        return set_error(CHEM_EUNSUPPORTED, "split-BF16 tables need %zu bytes of shared memory",
                         smem);
    if (t->fold)
        return t->nsp == 32 ? launch_nsp<32, true>(prm, smem, s, m->device)
                            : launch_nsp<64, true>(prm, smem, s, m->device);
    return t->nsp == 32 ? launch_nsp<32, false>(prm, smem, s, m->device)
                        : launch_nsp<64, false>(prm, smem, s, m->device);
}

}  // namespace chem
