// kern_bf16.cu -- split 16-bit source term on tcgen05 tensor cores (sm_103a).
//
// Per tile of 128 cells (one cell per tensor-memory lane), for reaction chunks of RC = 48
// (the last chunk holds the remaining 16..48 reactions):
//   contraction 1 (Eqs. 4, 6): S = A1 . [nu' | nu''] (M = 128, N = 2 RC, K = NSP), A1 =
//       [log2 z_k (k < ns), log2 c_tot, log2 c_tot - log2 sum_k z_k, Arrhenius features]
//       as two FP16 terms (hi + lo, 22 significant bits) in tensor memory.  The B rows are
//       the small-integer stoichiometric coefficients (exact in FP16), the third-body flag,
//       the reaction orders and the Arrhenius coefficients [log2 A, b, -E/R log2 e / 1000] on
//       the features [1, log2 T, 1000/T] (three FP16 rows each), so that S' = log2 q_f and
//       the reverse half = sum_k nu''_k log2 C_k + log2 k_f; an irreversible reaction's
//       reverse column and an empty slot carry a bias of -1e4 (2^S = 0).
//   Gibbs layer (Eqs. 8-11), folded per reaction: the reverse half also accumulates
//       -log2 K_c = sum_m c_mj phi_m(T) over 14 temperature features (NASA-7 terms
//       [1, log2 T, tau, tau^2, tau^3, tau^4, 1/tau], tau = T/1000, of the cell's
//       temperature range, the other range's seven zero), with c = nu^T . (per-species
//       coefficients) assembled in FP64 at load.  Features and coefficients are both two
//       FP16 terms; hi.hi, hi.lo and lo.hi are issued.  M = 128, N = RC, K = 16 per MMA.
//   epilogue (FP32, one thread per cell): q = 2^S' - 2^S'' (Eqs. 3-7); third-body factor
//       M / c_tot and falloff factor Pr / (1 + Pr) F (Sec. 2.4, the latter folded into the
//       exponents); q_net split into two BF16 terms (its range needs BF16's exponent)
//       written to one of two tensor-memory buffers.
//   contraction 2 (Eq. 2): omega += q_net . nu^T (M = 128, N = NSP, K = RC, BF16), in
//       tensor memory across the chunks; written once per tile.
//   contraction 0 (Sec. 2.4), once per tile: the third-body sums sum_k (eff_jk - 1) z_k of
//       the reactions that need them (M = 128, N = FCN, K = NSP), A = z as two BF16 terms
//       in the omega columns (free until contraction 2 of chunk 0), B = eff - 1 as two BF16
//       terms (hi.hi + hi.lo + lo.hi), into columns of their own read by the chunks that
//       hold those reactions.
//
// S and q_net have two tensor-memory buffers each: contraction 1 of chunk c + 1 runs while
// the epilogue works on chunk c, and the epilogue writes q_net of chunk c + 1 while
// contraction 2 of chunk c waits in the tensor pipe.  The next tile's operands are written
// during the last chunk (every contraction 1 of the current tile has completed by then), so
// its first contractions 1 run while the current omega is read out.
// Warp roles (480 threads): warp 0 bulk-copies the T, P, Y tile into shared memory;
// warp 1 owns tensor memory and issues contractions 1 from one thread, warp 14 issues
// contractions 0 and 2; warps 2-13 form three epilogue warpgroups, warpgroup g taking
// reactions 16 g .. 16 g + 15 of every chunk (warp w reaches tensor-memory lanes
// 32 (w % 4) .. 32 (w % 4) + 31).  Reactions with a third-body or falloff factor sit in the
// first 8 slots of "multiplier shares" (falloff ones in slots 0..3), each with 8 columns of
// third-body sums.
// Every mbarrier wait is bounded: on timeout the kernel records an error code in the
// mechanism's device status word and all roles wind down.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "chem_internal.h"
#include "kern_tc_common.cuh"
#include "tc_ptx.h"

namespace chem {

using namespace tck;

constexpr int kMaxFc = 64;             // third-body / falloff columns (8 per multiplier share)


struct Bf16Tables {
    int nsp, nch, rct, fcn;
    size_t blob_bytes;
    uint32_t o_bg, o_b2, o_e, o_qi, o_fq;   // offsets from the blob start
    void *d_blob;
    const uint16_t *btab;     // one contiguous block copied to shared memory
    const float *invW;
    int *status;
};

struct Bf16Params {
    const float *T, *P, *Y;
    float *om;
    int64_t n, ldY, ldO;
    int ns, nch, rct, fcn, ntiles;
    int stage_y;               // T, P, Y tiles staged in shared memory (the Y buffer then also
                               // stages omega on its way out)
    int bulk_out;              // omega rows contiguous (ldO == ns) and 16-byte aligned
    const uint16_t *btab;
    uint32_t blob_bytes;
    const float *invW;
    float t_mid, lg2R;
    int *status;
    // shared-memory layout (byte offsets from the 1024-aligned base); the copied block holds
    // B1, the Gibbs table, B2, the efficiency table, the share records and the falloff
    // records
    uint32_t o_bg, o_b2, o_e, o_qi, o_fq, o_y, o_t, o_p, o_iw, o_psum, o_bar;
};

enum {
    BAR_BTAB, BAR_YFULL, BAR_YEMPTY0, BAR_YEMPTY1, BAR_A1FULL, BAR_D1FULL0, BAR_D1FULL1, BAR_D1EMPTY0,
    BAR_D1EMPTY1, BAR_ZFULL, BAR_FCFULL, BAR_A2FULL0, BAR_A2FULL1, BAR_A2EMPTY0, BAR_A2EMPTY1,
    BAR_D2FULL, BAR_XREADY, BAR_DRAIN, BAR_COUNT
};

template <int NSP>
struct Cols {                                     // tensor-memory column map
    static constexpr uint32_t A1 = 0;             // contraction-1 operand: 2 terms x NSP/2
    static constexpr uint32_t AG = NSP;           // Gibbs features: 2 terms x 8
    static constexpr uint32_t S0 = ((AG + 16 + 31) / 32) * 32;   // two S buffers of 2 RC
    static constexpr uint32_t A2 = S0 + 4 * RC;   // two q_net buffers: 2 terms x RC/2 each
    static constexpr uint32_t FC = A2 + 2 * RC;   // third-body sums (contraction 0)
    static constexpr uint32_t D2 = FC + kMaxFc;   // omega; z (2 terms x NSP/2) at tile start
    static_assert(D2 + NSP <= kTmemCols, "tensor memory over budget");
};

template <int NSP>
__global__ void __launch_bounds__(kThreads, 1) k_source_bf16(const Bf16Params p)
{
    using CL = Cols<NSP>;
    // the prologue, z and omega columns are handled in blocks of 8, block i by warpgroup
    // i % NQ
    constexpr int NB = NSP / 8;
    constexpr int BPW = (NB + NQ - 1) / NQ;       // blocks per warpgroup, at most
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned base, offset on the shared array itself so that every access below
    // stays a shared-memory access (an integer round trip would make them generic)
    unsigned char *sm = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
    const uint32_t sbase = tc::smem_u32(sm);
    const QInfo *qinfo = (const QInfo *)(sm + p.o_qi);
    const FallQ *fallq = (const FallQ *)(sm + p.o_fq);
    float *Ys = (float *)(sm + p.o_y);
    float *Ts = (float *)(sm + p.o_t);
    float *Ps = (float *)(sm + p.o_p);
    float *Ws = (float *)(sm + p.o_y);            // omega [128][ns], in the Y buffer once the
                                                  // next tile's prologue has read it
    float *iW = (float *)(sm + p.o_iw);          // [NSP] 1 / W_k, zero past the species
    int *ccode = (int *)(iW + NSP);               // [NSP] what each contraction-1 column holds
    float *zrow = (float *)(ccode + NSP);         // [NSP] zeros: the Y row of a cell past n
    float *Psum = (float *)(sm + p.o_psum);      // [NQ][128] partial sums of z_k
    uint64_t *bars = (uint64_t *)(sm + p.o_bar);
    SmemCtl *ctl = (SmemCtl *)(bars + BAR_COUNT);
    auto BAR = [&](int i) { return tc::smem_u32(bars + i); };

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        constexpr uint32_t E = kEpiWarps;
        const uint32_t cnt[BAR_COUNT] = {1, 1, E, E, E, 1, 1, E, E, E, 1, E, E, 1, 1, 1, E, 2};
        for (int i = 0; i < BAR_COUNT; ++i) tc::mbar_init(BAR(i), cnt[i]);
        tc::mbar_fence_init();
        ctl->abort = 0;
    }
    if (warp == 1) {
        tc::tmem_alloc(tc::smem_u32(&ctl->tmem_base), kTmemCols);
        tc::tmem_relinquish();
    }
    for (int k = tid; k < NSP; k += kThreads) {
        iW[k] = k < p.ns ? p.invW[k] : 0.0f;
        zrow[k] = 0.0f;
        const int a = k - p.ns - 2;
        ccode[k] = k < p.ns ? kColSpecies : k == p.ns ? kColLgct : k == p.ns + 1 ? kColNorm
                 : (a >= 0 && a < kArrRows) ? kColOne + a / 3 : kColZero;
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = ctl->tmem_base;
    const int64_t n = p.n;
    const int nch = p.nch;

    if (warp == 0) {
        // ------------------------------------------------------------- tile loader
        if (lane == 0) {
            const uint32_t bt = p.blob_bytes;
            tc::mbar_arrive_expect_tx(BAR(BAR_BTAB), bt);
            for (uint32_t off = 0; off < bt; off += 16384)
                tc::bulk_g2s(sbase + off, (const unsigned char *)p.btab + off,
                             min(16384u, bt - off), BAR(BAR_BTAB));
            // The Y buffer holds Y of tile j from its load until the epilogue's prologue and z
            // have read it; then the omega of tile j - 1 is staged in it.  Event j (barrier
            // YEMPTY0 + (j & 1), its phase j >> 1): Y(j) read and omega(j - 1) staged (event 0:
            // Y(0) read); two barriers, so that the epilogue running two events ahead at the
            // end cannot alias a phase.  Before loading Y(j) this thread stores omega(j - 2)
            // and waits until the store has read the buffer.
            auto ywait = [&](int j) {
                return wait_bar(BAR(BAR_YEMPTY0 + (j & 1)), (j >> 1) & 1, ctl, p.status, 1);
            };
            auto bulk_tile = [&](int64_t i0) { return p.stage_y && p.bulk_out && i0 + 128 <= n; };
            auto store_omega = [&](int j) {           // omega of this CTA's tile j, if staged
                const int64_t i0 = (int64_t)(blockIdx.x + (int64_t)j * gridDim.x) * 128;
                if (j < 0 || !bulk_tile(i0)) return;
                tc::bulk_s2g(p.om + i0 * p.ldO, sbase + p.o_y, (uint32_t)(128 * p.ns * 4));
                tc::bulk_commit();
                tc::bulk_wait_read0();
            };
            int it = 0;
            bool pending = false, okl = true;
            for (int t = blockIdx.x; t < p.ntiles; t += gridDim.x, ++it) {
                if (it > 0) {
                    if (!(okl = ywait(it - 1))) break;
                    store_omega(it - 2);
                }
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
            // the last two tiles' omega
            if (okl && it > 0 && (okl = ywait(it - 1))) store_omega(it - 2);
            if (okl && it > 0 && ywait(it)) store_omega(it - 1);
            tc::bulk_wait0();                         // omega stores have landed
            // copies in flight are awaited before the CTA can exit
            if (pending && !okl) wait_bar(BAR(BAR_YFULL), (it - 1) & 1, ctl, p.status, 1);
            wait_bar(BAR(BAR_BTAB), 0, ctl, p.status, 1);
        }
    } else if (warp == 1 || warp == kMma2Warp) {
        // ------------------------------------------------------------- MMA issuers
        if (lane == 0) {
            constexpr uint32_t id2 = tc::idesc_bf16_f32(128, NSP);
            const uint32_t b1 = sbase, bg = sbase + p.o_bg, b2 = sbase + p.o_b2,
                           be = sbase + p.o_e;
            bool ok = wait_bar(BAR(BAR_BTAB), 0, ctl, p.status, 2);
            int it = 0;
            if (warp == 1) {
                // contraction 1 (+ the Gibbs layer) of each chunk into S buffer u & 1 as soon
                // as the epilogue has read that buffer's previous chunk
                uint32_t u = 0;
                for (int t = blockIdx.x; ok && t < p.ntiles; t += gridDim.x, ++it) {
                    if (!(ok = wait_bar(BAR(BAR_A1FULL), it & 1, ctl, p.status, 2))) break;
                    for (int c = 0; c < nch; ++c, ++u) {
                        const int b = (int)(u & 1);
                        if (!(ok = wait_bar(BAR(BAR_D1EMPTY0 + b), ((u >> 1) & 1) ^ 1, ctl,
                                            p.status, 2)))
                            break;
                        tc::fence_after();
                        const int rcc = c == nch - 1 ? p.rct : RC;
                        uint32_t d = tmem + CL::S0 + (uint32_t)b * (2 * RC), dr = d + rcc;
                        const uint32_t id1 = tc::idesc_f16_f32(128, 2 * rcc);
                        const uint32_t idg = tc::idesc_f16_f32(128, rcc);
                        const uint32_t bc = b1 + (uint32_t)c * (2 * RC * NSP * 2);
                        const uint32_t gc = bg + (uint32_t)c * (RC * kGibK * 2);
                        // every operand address before the burst of MMAs
                        uint64_t bd[NSP / 16], gd[2];
                        uint32_t aa[2][NSP / 16], ag[2];
#pragma unroll
                        for (int kk = 0; kk < NSP / 16; ++kk) {
                            bd[kk] = tc::sdesc_noswz(bc + kk * 256, 128, (NSP / 8) * 128);
                            aa[0][kk] = tmem + CL::A1 + kk * 8;
                            aa[1][kk] = tmem + CL::A1 + NSP / 2 + kk * 8;
                            tc::pin(bd[kk]);
                            tc::pin(aa[0][kk]);
                            tc::pin(aa[1][kk]);
                        }
#pragma unroll
                        for (int tt = 0; tt < 2; ++tt) {
                            gd[tt] = tc::sdesc_noswz(gc + tt * 256, 128, (kGibK / 8) * 128);
                            ag[tt] = tmem + CL::AG + tt * 8;
                            tc::pin(gd[tt]);
                            tc::pin(ag[tt]);
                        }
                        tc::pin(d);
                        tc::pin(dr);
#pragma unroll
                        for (int s = 0; s < 2; ++s)
#pragma unroll
                            for (int kk = 0; kk < NSP / 16; ++kk)
                                tc::mma_ts(d, aa[s][kk], bd[kk], id1, (s | kk) != 0);
                        // Gibbs layer into the reverse half: feature term s against the
                        // coefficient terms 0 .. 1 - s
#pragma unroll
                        for (int s = 0; s < 2; ++s)
#pragma unroll
                            for (int tt = 0; tt < 2 - s; ++tt) tc::mma_ts(dr, ag[s], gd[tt], idg, 1);
                        tc::commit(BAR(BAR_D1FULL0 + b));
                    }
                }
            } else {
                // per tile: contraction 0 once z is in the omega columns (ZFULL: the tile
                // before's omega has been read out and the third-body sums of its last
                // chunks as well), then contraction 2 of each chunk in chunk order (the
                // accumulation order, hence the rounding, is fixed)
                const uint32_t id0 = tc::idesc_bf16_f32(128, p.fcn);
                uint32_t u = 0;
                for (int t = blockIdx.x; ok && t < p.ntiles; t += gridDim.x, ++it) {
                    if (!(ok = wait_bar(BAR(BAR_ZFULL), it & 1, ctl, p.status, 2))) break;
                    tc::fence_after();
                    {
                        uint64_t ed[2][NSP / 16];
                        uint32_t za[2][NSP / 16], dfc = tmem + CL::FC;
#pragma unroll
                        for (int kk = 0; kk < NSP / 16; ++kk) {
                            ed[0][kk] = tc::sdesc_noswz(be + kk * 256, 128, (NSP / 8) * 128);
                            ed[1][kk] = tc::sdesc_noswz(be + p.fcn * NSP * 2 + kk * 256, 128, (NSP / 8) * 128);
                            za[0][kk] = tmem + CL::D2 + kk * 8;
                            za[1][kk] = tmem + CL::D2 + NSP / 2 + kk * 8;
                            tc::pin(ed[0][kk]);
                            tc::pin(ed[1][kk]);
                            tc::pin(za[0][kk]);
                            tc::pin(za[1][kk]);
                        }
                        tc::pin(dfc);
                        // z hi . E hi, z hi . E lo, z lo . E hi
#pragma unroll
                        for (int s = 0; s < 3; ++s)
#pragma unroll
                            for (int kk = 0; kk < NSP / 16; ++kk)
                                tc::mma_ts(dfc, za[s == 2][kk], ed[s == 1][kk], id0, (s | kk) != 0);
                    }
                    tc::commit(BAR(BAR_FCFULL));
                    for (int c = 0; c < nch; ++c, ++u) {
                        const int ab = (int)(u & 1);
                        if (!(ok = wait_bar(BAR(BAR_A2FULL0 + ab), (u >> 1) & 1, ctl, p.status, 2)))
                            break;
                        tc::fence_after();
                        const int rcc = c == nch - 1 ? p.rct : RC;
                        const int nk = rcc / 16;
                        const uint32_t bc = b2 + (uint32_t)c * (NSP * RC * 2);
                        const uint32_t a2 = tmem + CL::A2 + (uint32_t)ab * RC;
                        uint64_t bd[RC / 16];
                        uint32_t aa[2][RC / 16], dd = tmem + CL::D2;
#pragma unroll
                        for (int kk = 0; kk < RC / 16; ++kk) {
                            bd[kk] = tc::sdesc_noswz(bc + kk * 256, 128, (rcc / 8) * 128);
                            aa[0][kk] = a2 + kk * 8;
                            aa[1][kk] = a2 + RC / 2 + kk * 8;
                            tc::pin(bd[kk]);
                            tc::pin(aa[0][kk]);
                            tc::pin(aa[1][kk]);
                        }
                        tc::pin(dd);
#pragma unroll
                        for (int s = 0; s < 2; ++s)
#pragma unroll
                            for (int kk = 0; kk < RC / 16; ++kk)
                                if (kk < nk) tc::mma_ts(dd, aa[s][kk], bd[kk], id2, (c | s | kk) != 0);
                        tc::commit(BAR(BAR_A2EMPTY0 + ab));
                    }
                    if (ok) tc::commit(BAR(BAR_D2FULL));
                }
            }
            // every MMA issued (by both issuers) has completed before tensor memory is released
            tc::commit(BAR(BAR_DRAIN));
            wait_bar(BAR(BAR_DRAIN), 0, ctl, p.status, 2);
        }
    } else if (warp < kMma2Warp) {
        // ------------------------------------------------------------- epilogue
        const int ew = warp - kEpiWarp0;             // 0 .. kEpiWarps - 1
        const int g = ew >> 2;                        // warpgroup: share of each chunk
        const int q = warp & 3;                       // lane quarter of tensor memory
        const int row = q * 32 + lane;
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        const int ns = p.ns;
        int it = 0;
        uint32_t u = 0;
        bool ok = wait_bar(BAR(BAR_BTAB), 0, ctl, p.status, 3);   // tables in smem
        CellF cf;
        // this thread's species row of tile t: staged in shared memory (full tiles) or read
        // from global memory
        auto y_row = [&](int t) -> const float * {
            const int64_t i0 = (int64_t)t * 128, ci = i0 + row;
            if (p.stage_y && i0 + 128 <= n) return Ys + (int64_t)row * p.ldY;
            return ci < n ? p.Y + ci * p.ldY : zrow;
        };
        // ---- prologue of tile t: features, z, split log2 z (Eq. 4 input layer), the
        // Arrhenius and Gibbs features; ends with contraction 1's operands in tensor memory
        // (A1FULL)
        auto prologue = [&](int t, int itp, CellF &cf) -> bool {
            const int64_t i0 = (int64_t)t * 128;
            const int64_t ci = i0 + row;
            const bool full = p.stage_y && i0 + 128 <= n;
            if (!wait_bar(BAR(BAR_YFULL), itp & 1, ctl, p.status, 3)) return false;
            float Tc = 1000.0f, Pc = 1.0e6f;
            if (full) {
                Tc = Ts[row];
                Pc = Ps[row];
            } else if (ci < n) {
                Tc = __ldg(p.T + ci);
                Pc = __ldg(p.P + ci);
            }
            const float *yrow = y_row(t);
            cf.lg2T = log2f(Tc);
            cf.invT = 1.0f / Tc;
            cf.itau = 1000.0f / Tc;
            cf.T = Tc;
            cf.lgct = log2f(Pc) - p.lg2R - cf.lg2T;
            // this warpgroup's blocks of columns: z_k = Y_k / W_k (species), whose log2 goes
            // to the contraction; X_k = z_k / sum_k z_k is completed by column ns + 1
            // (log2 c_tot - log2 sum_k z_k, weighted by the reaction order), written once the
            // warpgroups' partial sums are in.  Every contraction 1 of the previous tile has
            // completed (the epilogue waited for the last one's D1FULL), so A1 and AG are free
            // and each block goes to tensor memory as soon as it is formed.
            tc::fence_after();
            float psum = 0.0f;
#pragma unroll
            for (int bi = 0; bi < BPW; ++bi) {
                const int blk = g + NQ * bi;
                if (blk >= NB) continue;
                float lx[8];
                const float4 w0 = *(const float4 *)(iW + 8 * blk), w1 = *(const float4 *)(iW + 8 * blk + 4);
                const float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
                if (8 * blk + 8 <= ns) {
                    // species only (straight-line, so that the loads and logarithms overlap)
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const float z = fmaxf(yrow[8 * blk + e], 0.0f) * wv[e];
                        psum += z;
                        lx[e] = fmaxf(tc::lg2(z), kLog2Floor);
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        // loads clamped to the row, z = 0 past the species
                        const int k = 8 * blk + e;
                        const float z = fmaxf(yrow[min(k, ns - 1)], 0.0f) * wv[e];
                        psum += z;
                        const float lz = fmaxf(tc::lg2(z), kLog2Floor);
                        const int cc = ccode[k];
                        // species, the third-body c_tot column, the Arrhenius features 1,
                        // log2 T, 1000/T (each against three coefficient rows); the
                        // normalisation later
                        lx[e] = cc == kColSpecies ? lz : cc == kColLgct ? cf.lgct
                              : cc == kColOne ? 1.0f : cc == kColLg2T ? cf.lg2T
                              : cc == kColItau ? cf.itau : 0.0f;
                    }
                }
                uint32_t wh[4], wl[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) split2h(lx[2 * e], lx[2 * e + 1], wh[e], wl[e]);
                const uint32_t a1 = tmem + lane_off + CL::A1 + 4 * blk;
                tc::tmem_st4(a1, wh);
                tc::tmem_st4(a1 + NSP / 2, wl);
            }
            Psum[g * 128 + row] = psum;
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(BAR(BAR_XREADY));
            if (g == NQ - 1) {
                // Gibbs features: NASA-7 terms of the cell's temperature range
                const float tau = Tc * 1e-3f, t2 = tau * tau;
                const float ph[7] = {1.0f, cf.lg2T, tau, t2, t2 * tau, t2 * t2, cf.itau};
                const bool hi = Tc >= p.t_mid;
                float fv[16];
#pragma unroll
                for (int m = 0; m < 7; ++m) {
                    fv[m] = hi ? 0.0f : ph[m];
                    fv[7 + m] = hi ? ph[m] : 0.0f;
                }
                fv[14] = fv[15] = 0.0f;
                uint32_t gh[8], gl[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) split2h(fv[2 * e], fv[2 * e + 1], gh[e], gl[e]);
                const uint32_t ag = tmem + lane_off + CL::AG;
                tc::tmem_st8(ag + 0, gh);
                tc::tmem_st8(ag + 8, gl);
            }
            if (!wait_bar(BAR(BAR_XREADY), itp & 1, ctl, p.status, 3)) return false;
            float sum = 0.0f;
#pragma unroll
            for (int gg = 0; gg < NQ; ++gg) sum += Psum[gg * 128 + row];
            cf.inv_sum = sum > 0.0f ? 1.0f / sum : 0.0f;
            {
                // the packed word holding the normalisation column ns + 1 and its neighbour
                // (column ns, log2 c_tot, or ns + 2, the Arrhenius feature 1 or padding)
                const int kn = ns + 1;
                tc::tmem_wait_st();                   // the block holding it has landed
                if ((kn >> 3) % NQ == g) {
                    const float vn = sum > 0.0f ? cf.lgct - log2f(sum) : 0.0f;
                    const int ko = kn ^ 1;
                    const int co = ccode[ko];
                    const float vo = co == kColLgct ? cf.lgct : co == kColOne ? 1.0f : 0.0f;
                    const float lo = (kn & 1) ? vo : vn, hi = (kn & 1) ? vn : vo;
                    uint32_t h, l;
                    split2h(lo, hi, h, l);
                    const uint32_t col = tmem + lane_off + CL::A1 + kn / 2;
                    tc::tmem_st1(col, h);
                    tc::tmem_st1(col + NSP / 2, l);
                }
            }
            tc::tmem_wait_st();
            tc::fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(BAR(BAR_A1FULL));
            return true;
        };
        // z of tile t (two BF16 terms, contraction 0's operand) into the omega columns once
        // the tile before's omega has been read out; recomputed from the tile's Y, which
        // that omega has not yet replaced in the staging buffer
        auto write_z = [&](int t) {
            const float *yrow = y_row(t);
#pragma unroll
            for (int bi = 0; bi < BPW; ++bi) {
                if (g + NQ * bi >= NB) continue;
                const int blk = g + NQ * bi;
                const float4 w0 = *(const float4 *)(iW + 8 * blk), w1 = *(const float4 *)(iW + 8 * blk + 4);
                const float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
                float zz[8];
                if (8 * blk + 8 <= ns) {
#pragma unroll
                    for (int e = 0; e < 8; ++e) zz[e] = fmaxf(yrow[8 * blk + e], 0.0f) * wv[e];
                } else {
#pragma unroll
                    for (int e = 0; e < 8; ++e) zz[e] = fmaxf(yrow[min(8 * blk + e, ns - 1)], 0.0f) * wv[e];
                }
                uint32_t zh[4], zl[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) split2x2(zz[2 * e], zz[2 * e + 1], zh[e], zl[e]);
                const uint32_t az = tmem + lane_off + CL::D2 + 4 * (g + NQ * bi);
                tc::tmem_st4(az, zh);
                tc::tmem_st4(az + NSP / 2, zl);
            }
            tc::tmem_wait_st();
        };
        if ((int)blockIdx.x < p.ntiles) {
            ok = ok && prologue(blockIdx.x, 0, cf);
            if (ok) {
                write_z(blockIdx.x);
                tc::fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(BAR(BAR_ZFULL));
                if (lane == 0) tc::mbar_arrive(BAR(BAR_YEMPTY0));   // event 0: Y(0) read
            }
        }
        CellF cfn;                                    // features of the next tile
        for (int t = blockIdx.x; ok && t < p.ntiles; t += gridDim.x, ++it) {
            const int64_t i0 = (int64_t)t * 128;
            const int64_t ci = i0 + row;
            const int t_next = t + gridDim.x;
            const bool has_next = t_next < p.ntiles;
            bool fc_ready = false;
            // ---- every chunk, this warpgroup's share of its reactions.  The S read-out of
            // chunk c + 1 is issued before chunk c's q_net goes out, so that its latency
            // overlaps that store.
            uint32_t sf[RH], sr[RH];
            auto load_s = [&](int c, uint32_t uu) -> bool {
                const int b = (int)(uu & 1);
                if (!wait_bar(BAR(BAR_D1FULL0 + b), (uu >> 1) & 1, ctl, p.status, 3)) return false;
                tc::fence_after();
                const int rcc = c == nch - 1 ? p.rct : RC;
                if (g * RH < rcc) {
                    const uint32_t d1 = tmem + lane_off + CL::S0 + (uint32_t)b * (2 * RC) + g * RH;
                    tc::tmem_ld16_nw(d1, sf);
                    tc::tmem_ld16_nw(d1 + rcc, sr);
                }
                return true;
            };
            auto release_s = [&](int c, uint32_t uu) {
                const int rcc = c == nch - 1 ? p.rct : RC;
                if (g * RH < rcc) tc::tmem_wait_ld_tie16(sf, sr);
                tc::fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(BAR(BAR_D1EMPTY0 + (int)(uu & 1)));
            };
            if (!(ok = load_s(0, u))) break;
            release_s(0, u);
            for (int c = 0; c < nch; ++c, ++u) {
                const int rcc = c == nch - 1 ? p.rct : RC;
                const bool active = g * RH < rcc;
                const QInfo qi = qinfo[c * NQ + g];
                float qv[RH];
                if (active) {
                    if (qi.rank >= 0) {
                        // the share's third-body / falloff reactions sit in its first 8 slots
                        // (falloff in 0..nfall-1); their columns hold sum_k (eff_k - 1) z_k
                        // (0 for plain slots), so M / c_tot = 1 + that / sum_k z_k
                        if (!fc_ready) {
                            if (!(ok = wait_bar(BAR(BAR_FCFULL), it & 1, ctl, p.status, 3))) break;
                            tc::fence_after();
                            fc_ready = true;
                        }
                        uint32_t fv[8];
                        tc::tmem_ld8(tmem + lane_off + CL::FC + 8 * qi.rank, fv);
                        float s8[8], fac[4], mul[4];
#pragma unroll
                        for (int r = 0; r < 8; ++r) s8[r] = fmaf(__uint_as_float(fv[r]), cf.inv_sum, 1.0f);
                        falloff4(fallq + 4 * qi.rank, s8, cf, qi.nfall, fac, mul);
#pragma unroll
                        for (int r = 0; r < 4; ++r)
                            qv[r] = (tc::ex2(__uint_as_float(sf[r]) + fac[r]) -
                                     tc::ex2(__uint_as_float(sr[r]) + fac[r])) * mul[r];
#pragma unroll
                        for (int r = 4; r < 8; ++r)
                            qv[r] = (tc::ex2(__uint_as_float(sf[r])) -
                                     tc::ex2(__uint_as_float(sr[r]))) * s8[r];
#pragma unroll
                        for (int r = 8; r < RH; ++r)
                            qv[r] = tc::ex2(__uint_as_float(sf[r])) - tc::ex2(__uint_as_float(sr[r]));
                    } else {
#pragma unroll
                        for (int r = 0; r < RH; ++r)
                            qv[r] = tc::ex2(__uint_as_float(sf[r])) - tc::ex2(__uint_as_float(sr[r]));
                    }
                }
                uint32_t hw[RH / 2], lw[RH / 2];
                if (active) {
#pragma unroll
                    for (int r = 0; r < RH; r += 2) split2x2(qv[r], qv[r + 1], hw[r / 2], lw[r / 2]);
                }
                // next chunk's S read-out in flight during this chunk's store
                if (c + 1 < nch && !(ok = load_s(c + 1, u + 1))) break;
                const int ab = (int)(u & 1);
                if (!(ok = wait_bar(BAR(BAR_A2EMPTY0 + ab), ((u >> 1) & 1) ^ 1, ctl, p.status, 3))) break;
                tc::fence_after();
                if (active) {
                    const uint32_t a2 = tmem + lane_off + CL::A2 + (uint32_t)ab * RC + g * (RH / 2);
                    tc::tmem_st8(a2, hw);
                    tc::tmem_st8(a2 + RC / 2, lw);
                    tc::tmem_wait_st();
                }
                tc::fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(BAR(BAR_A2FULL0 + ab));
                // last chunk: every contraction 1 of this tile has completed, so the next
                // tile's prologue writes its operands now; its contractions 1 run while this
                // chunk's contraction 2 and the omega read-out finish
                if (c == nch - 1 && has_next && !(ok = prologue(t_next, it + 1, cfn))) break;
                if (c + 1 < nch) release_s(c + 1, u + 1);
            }
            if (!ok) break;
            // ---- omega of the tile: tensor memory -> registers; then the next tile's z
            // into the omega columns and ZFULL (z ready; this tile's third-body sums, read
            // by its chunks, may be replaced)
            if (!(ok = wait_bar(BAR(BAR_D2FULL), it & 1, ctl, p.status, 3))) break;
            tc::fence_after();
            uint32_t w[BPW][8];
#pragma unroll
            for (int bi = 0; bi < BPW; ++bi)
                if (g + NQ * bi < NB) tc::tmem_ld8(tmem + lane_off + CL::D2 + 8 * (g + NQ * bi), w[bi]);
            if (has_next) write_z(t_next);
            tc::fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(BAR(BAR_ZFULL));
            // ---- omega -> shared (the Y buffer, read by the next tile's prologue and z
            // already), stored by the loader thread; partial tiles and padded rows go out
            // directly
            if (p.stage_y && p.bulk_out && i0 + 128 <= n) {
#pragma unroll
                for (int bi = 0; bi < BPW; ++bi)
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int k = 8 * (g + NQ * bi) + e;
                        if (k < ns) Ws[row * ns + k] = __uint_as_float(w[bi][e]);
                    }
                tc::fence_proxy_async_smem();            // visible to the bulk store
            } else if (ci < n) {
                float *orow = p.om + ci * p.ldO;
#pragma unroll
                for (int bi = 0; bi < BPW; ++bi)
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int k = 8 * (g + NQ * bi) + e;
                        if (k < ns) orow[k] = __uint_as_float(w[bi][e]);
                    }
            }
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(BAR(BAR_YEMPTY0 + ((it + 1) & 1)));   // event it + 1
            cf = cfn;
        }
    }
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

chem_status wide_build_tables(chem_mech *m, const chem_mech_desc *d, void **out);
void wide_free_tables(void *p);
int *wide_status_word(const void *p);
chem_status wide_check(const void *p);
chem_status launch_source_wide(const chem_mech *m, const void *tables, int64_t n, const float *T,
                               const float *P, const float *Y, int64_t ldY, float *om, int64_t ldO,
                               cudaStream_t s);

chem_status bf16_build_tables(chem_mech *m, const chem_mech_desc *d)
{
    const int ns = d->n_species, nr = d->n_reactions;
    // contraction-1 columns: species 0..ns-1, log2 c_tot (third-body factor), the
    // normalisation column log2 c_tot - log2 sum_k z_k (weighted by the reaction order), and
    // the nine Arrhenius rows
    int nsp = ns + 2 + kArrRows;
    if (nsp <= 32) nsp = 32;
    else if (nsp <= 64) nsp = 64;
    else {
        // larger mechanisms: operands in shared memory, tables streamed (kern_wide.cu)
        void *w = nullptr;
        chem_status st = wide_build_tables(m, d, &w);
        if (st != CHEM_OK) return st;
        st = wide_check(w);
        if (st != CHEM_OK) {
            wide_free_tables(w);
            return st;
        }
        m->bf16 = w;
        m->bf16_wide = true;
        m->have_bf16 = true;
        return CHEM_OK;
    }
    const int kf0 = ns + 2;
    const int nrp = ((nr + 15) / 16) * 16;
    const int nch = (nrp + RC - 1) / RC;
    const int rct = nrp - (nch - 1) * RC;      // reactions of the last chunk, 16..RC
    // chunk shares (chunk, warpgroup) of RH slots; multiplier shares are taken from the end,
    // chunk 0 last (its multipliers would have to wait for contraction 0)
    std::vector<int> plain, fall, tbr;
    for (int j = 0; j < nr; ++j)
        (d->kind[j] == 0 ? plain : d->kind[j] == CHEM_RXN_THIRD_BODY ? tbr : fall).push_back(j);
    const int nspec = (int)(fall.size() + tbr.size());
    int qm = 0;
    if (nspec) qm = std::max((nspec + 7) / 8, ((int)fall.size() + 3) / 4);
    std::vector<int> shares;                   // c * NQ + g, in the order they are taken
    for (int c = nch - 1; c >= 1; --c)
        for (int gq = (c == nch - 1 ? rct / RH : NQ) - 1; gq >= 0; --gq) shares.push_back(c * NQ + gq);
    for (int gq = (nch == 1 ? rct / RH : NQ) - 1; gq >= 0; --gq) shares.push_back(gq);
    const int fcn = std::max(16, ((8 * qm + 15) / 16) * 16);
    if (qm > (int)shares.size() || fcn > kMaxFc)
        return set_error(CHEM_EUNSUPPORTED,
                         "split-BF16 path: %d third-body / falloff reactions (%d falloff) exceed "
                         "its %d multiplier columns", nspec, (int)fall.size(), kMaxFc);
    std::vector<QInfo> qinfo((size_t)nch * NQ);
    for (auto &x : qinfo) x = QInfo{-1, 0, 0, 0};
    std::vector<int> qsel(shares.begin(), shares.begin() + qm);
    std::sort(qsel.begin(), qsel.end());       // ascending chunk order
    for (int r = 0; r < qm; ++r) qinfo[qsel[r]].rank = (int8_t)r;
    // slot -> reaction (-1: empty): falloff round-robin into slots 0..3 of the multiplier
    // shares, third-body into the least filled, then the plain reactions in order
    std::vector<int> order((size_t)nch * RC, -1);
    auto slot_of = [&](int qq, int pos) { return (qq / NQ) * RC + (qq % NQ) * RH + pos; };
    {
        std::vector<int> fill(qm, 0);
        for (size_t i = 0; i < fall.size(); ++i) {
            const int r = (int)(i % qm);
            order[slot_of(qsel[r], fill[r]++)] = fall[i];
        }
        for (int r = 0; r < qm; ++r) qinfo[qsel[r]].nfall = (int8_t)fill[r];
        for (size_t i = 0; i < tbr.size(); ++i) {
            int r = 0;
            for (int x = 1; x < qm; ++x)
                if (fill[x] < fill[r]) r = x;
            if (fill[r] >= 8)
                return set_error(CHEM_EUNSUPPORTED, "split-BF16 path: multiplier slot layout");
            order[slot_of(qsel[r], fill[r]++)] = tbr[i];
        }
        size_t pi = 0;
        for (int c = 0; c < nch && pi < plain.size(); ++c)
            for (int r = 0; r < (c == nch - 1 ? rct : RC) && pi < plain.size(); ++r)
                if (order[(size_t)c * RC + r] < 0) order[(size_t)c * RC + r] = plain[pi++];
        if (pi != plain.size()) return set_error(CHEM_EUNSUPPORTED, "split-BF16 path: slot layout");
    }
    // tables: B1 [chunk][2 rcc][nsp], BG [chunk][rcc][48], B2 [chunk][nsp][rcc] (core-matrix
    // order, K-major), E [term][fcn][nsp]; each chunk at the stride of a full one
    const size_t b1c = (size_t)2 * RC * nsp, bgc = (size_t)RC * kGibK, b2c = (size_t)nsp * RC;
    std::vector<uint16_t> b1(b1c * nch, 0), bgt(bgc * nch, 0), b2(b2c * nch, 0);
    const size_t e_term = (size_t)fcn * nsp;
    std::vector<uint16_t> eb(2 * e_term, 0);
    auto b1_at = [&](int c, int rcc, int r, int k) -> uint16_t & {
        (void)rcc;
        return b1[(size_t)c * b1c + ((r / 8) * (nsp / 8) + k / 8) * 64 + (r % 8) * 8 + k % 8];
    };
    auto bg_at = [&](int c, int r, int k) -> uint16_t & {
        return bgt[(size_t)c * bgc + ((r / 8) * (kGibK / 8) + k / 8) * 64 + (r % 8) * 8 + k % 8];
    };
    auto b2_at = [&](int c, int rcc, int nrow, int r) -> uint16_t & {
        return b2[(size_t)c * b2c + ((nrow / 8) * (rcc / 8) + r / 8) * 64 + (nrow % 8) * 8 + r % 8];
    };
    auto e_at = [&](int term, int col, int k) -> uint16_t & {
        return eb[term * e_term + ((col / 8) * (nsp / 8) + k / 8) * 64 + (col % 8) * 8 + k % 8];
    };
    // Gibbs layer per species on [1, log2 T, tau, tau^2, tau^3, tau^4, 1/tau] (tau = T/1000)
    // in log2 units, the standard concentration folded into the bias (Eqs. 10-11):
    // G = (a1 - a7) log2e - log2(p_ref/R) + (1 - a1) log2 T - a2/2 T log2e - a3/6 T^2 log2e
    //     - a4/12 T^3 log2e - a5/20 T^4 log2e + a6 log2e / T
    const double lg2_pref_R = log2(d->p_ref / kR);
    std::vector<double> gsp((size_t)ns * 14);
    for (int k = 0; k < ns; ++k)
        for (int rg = 0; rg < 2; ++rg) {
            const double *a = d->nasa7 + (size_t)k * 14 + (size_t)rg * 7;
            const double cc[7] = {(a[0] - a[6]) * kLog2e - lg2_pref_R, 1.0 - a[0],
                                  -a[1] / 2.0 * 1e3 * kLog2e, -a[2] / 6.0 * 1e6 * kLog2e,
                                  -a[3] / 12.0 * 1e9 * kLog2e, -a[4] / 20.0 * 1e12 * kLog2e,
                                  a[5] * kLog2e * 1e-3};
            for (int q = 0; q < 7; ++q) gsp[(size_t)k * 14 + rg * 7 + q] = cc[q];
        }
    FallQ neutral;
    memset(&neutral, 0, sizeof neutral);
    neutral.troe = make_float4(1.0f, 0.0f, 0.0f, 0.0f);
    neutral.t2 = make_float4(1e30f, 0.0f, 0.0f, 0.0f);
    std::vector<FallQ> fq((size_t)std::max(qm, 1) * 4, neutral);
    std::vector<int> qrank((size_t)nch * NQ, -1);
    for (int r = 0; r < qm; ++r) qrank[qsel[r]] = r;
    for (int c = 0; c < nch; ++c) {
        const int rcc = c == nch - 1 ? rct : RC;
        for (int r = 0; r < rcc; ++r) {
            const int j = order[(size_t)c * RC + r];
            uint16_t dead[3];
            f16_split<3>(kDead, dead);
            if (j < 0) {                          // padding slot: q = 0
                for (int i = 0; i < 3; ++i) b1_at(c, rcc, r, kf0 + i) = b1_at(c, rcc, rcc + r, kf0 + i) = dead[i];
                continue;
            }
            const int kind = d->kind[j];
            const double *ar = d->arrh + (size_t)j * 3;
            int ordf = 0, ordr = 0;
            for (int k = 0; k < ns; ++k) {
                const int f = d->nu_f[(size_t)j * ns + k], pr = d->nu_r[(size_t)j * ns + k];
                ordf += f;
                ordr += pr;
                b1_at(c, rcc, r, k) = f16_of_int(f);
                b1_at(c, rcc, rcc + r, k) = f16_of_int(pr);
                b2_at(c, rcc, k, r) = bf16_of_int(pr - f);
            }
            const int tbx = kind == CHEM_RXN_THIRD_BODY ? 1 : 0;   // log2 M = log2 c_tot + log2(M/c_tot)
            b1_at(c, rcc, r, ns) = f16_of_int(tbx);
            b1_at(c, rcc, rcc + r, ns) = f16_of_int(tbx);
            b1_at(c, rcc, r, ns + 1) = f16_of_int(ordf);
            b1_at(c, rcc, rcc + r, ns + 1) = f16_of_int(ordr);
            // rows kf0 + 3 f + i: term i of the coefficient of feature f (1, log2 T, 1000/T)
            const double co[3] = {ar[0] * kLog2e, ar[1], -ar[2] * kLog2e * 1e-3};
            for (int f = 0; f < 3; ++f) {
                uint16_t t3[3];
                f16_split<3>(co[f], t3);
                for (int i = 0; i < 3; ++i) {
                    b1_at(c, rcc, r, kf0 + 3 * f + i) = t3[i];
                    if (d->reversible[j]) b1_at(c, rcc, rcc + r, kf0 + 3 * f + i) = t3[i];
                }
            }
            if (!d->reversible[j])
                for (int i = 0; i < 3; ++i) b1_at(c, rcc, rcc + r, kf0 + i) = dead[i];
            else {
                // Gibbs layer folded through nu (FP64): coefficient of feature m of range rg
                for (int rg = 0; rg < 2; ++rg)
                    for (int q = 0; q < 7; ++q) {
                        double cj = 0.0;
                        for (int k = 0; k < ns; ++k) {
                            const int nu = d->nu_r[(size_t)j * ns + k] - d->nu_f[(size_t)j * ns + k];
                            if (nu) cj += nu * gsp[(size_t)k * 14 + rg * 7 + q];
                        }
                        uint16_t t2[2];
                        f16_split<2>(cj, t2);
                        for (int i = 0; i < 2; ++i) bg_at(c, r, 16 * i + 7 * rg + q) = t2[i];
                    }
            }
            if (kind == 0) continue;
            // third-body sum column (contraction 0): eff - 1 in two BF16 terms
            const int qq = c * NQ + r / RH, pos = r % RH;
            const int rk = qrank[qq];
            if (rk < 0 || pos >= 8 || (kind != CHEM_RXN_THIRD_BODY && pos >= 4))
                return set_error(CHEM_EUNSUPPORTED, "split-BF16 path: multiplier slot layout");
            const int col = 8 * rk + pos;
            for (int k = 0; k < ns; ++k) {
                const double e = (d->eff ? d->eff[(size_t)j * ns + k] : 1.0) - 1.0;
                const uint16_t hi = bf16_rn((float)e);
                e_at(0, col, k) = hi;
                e_at(1, col, k) = bf16_rn((float)(e - f_of_bf16(hi)));
            }
            if (kind != CHEM_RXN_THIRD_BODY) {
                FallQ &F = fq[(size_t)4 * rk + pos];
                const double *al = d->arrh_low + (size_t)j * 3;
                F.kf = make_float4((float)co[0], (float)co[1], (float)(-ar[2] * kLog2e), 1.0f);
                F.k0 = make_float4((float)(al[0] * kLog2e), (float)al[1], (float)(-al[2] * kLog2e), 0.f);
                if (kind == CHEM_RXN_TROE) {
                    const double *tp = d->troe + (size_t)j * 4;
                    F.troe = make_float4((float)(1.0 - tp[0]), (float)tp[0], (float)(kLog2e / tp[1]),
                                         (float)(kLog2e / tp[2]));
                    if (tp[3] > 0.0) F.t2 = make_float4((float)(tp[3] * kLog2e), 0, 0, 0);
                }
            }
        }
    }
    std::vector<float> invW(ns);
    for (int k = 0; k < ns; ++k) invW[k] = (float)(1.0 / d->mol_weight[k]);

    // B1 | BG | B2 | E | share records | falloff: contiguous, copied to
    // shared memory by bulk transfers (16-byte granules); the last chunk of each table is
    // cut to its rows
    auto a16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
    auto a256 = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t sb1 = (b1c * (nch - 1) + (size_t)2 * rct * nsp) * 2;
    const size_t sbg = (bgc * (nch - 1) + (size_t)rct * kGibK) * 2;
    const size_t sb2 = (b2c * (nch - 1) + (size_t)nsp * rct) * 2;
    const size_t ob1 = 0, obg = a16(ob1 + sb1), ob2 = a16(obg + sbg), oe = a16(ob2 + sb2);
    const size_t oqi = a16(oe + eb.size() * 2);
    const size_t ofq = a16(oqi + qinfo.size() * sizeof(QInfo));
    const size_t blob = a16(ofq + fq.size() * sizeof(FallQ));
    const size_t oiw = a256(blob), ost = a256(oiw + invW.size() * 4), total = a256(ost + 16);
    std::vector<unsigned char> h(total, 0);
    memcpy(h.data() + ob1, b1.data(), sb1);
    memcpy(h.data() + obg, bgt.data(), sbg);
    memcpy(h.data() + ob2, b2.data(), sb2);
    memcpy(h.data() + oe, eb.data(), eb.size() * 2);
    memcpy(h.data() + oqi, qinfo.data(), qinfo.size() * sizeof(QInfo));
    memcpy(h.data() + ofq, fq.data(), fq.size() * sizeof(FallQ));
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
    t->nch = nch;
    t->rct = rct;
    t->fcn = fcn;
    t->blob_bytes = blob;
    t->o_bg = (uint32_t)obg;
    t->o_b2 = (uint32_t)ob2;
    t->o_e = (uint32_t)oe;
    t->o_qi = (uint32_t)oqi;
    t->o_fq = (uint32_t)ofq;
    t->btab = (const uint16_t *)(base + ob1);
    t->invW = (const float *)(base + oiw);
    t->status = (int *)(base + ost);
    m->bf16 = t;
    m->have_bf16 = true;
    m->device_bytes += total;
    return CHEM_OK;
}

void bf16_free_tables(chem_mech *m)
{
    if (!m->bf16) return;
    if (m->bf16_wide) {
        wide_free_tables(m->bf16);
    } else {
        Bf16Tables *t = (Bf16Tables *)m->bf16;
        cudaFree(t->d_blob);
        delete t;
    }
    m->bf16 = nullptr;
}

int *bf16_status_word(const chem_mech *m)
{
    if (!m->have_bf16) return nullptr;
    return m->bf16_wide ? wide_status_word(m->bf16) : ((Bf16Tables *)m->bf16)->status;
}

template <int NSP>
static chem_status launch_nsp(const Bf16Params &prm, size_t smem, cudaStream_t s, int dev)
{
    static SmemOptIn opt;
    const int grid = std::min(prm.ntiles, sm_limit(sm_count(dev)));
    chem_status st = launch_opted(opt, (const void *)k_source_bf16<NSP>, 227 * 1024, "split-BF16",
                                  [&] { k_source_bf16<NSP><<<grid, kThreads, smem, s>>>(prm); });
    if (st == CHEM_OK) g_launches.fetch_add(1);
    return st;
}

chem_status launch_source_bf16(const chem_mech *m, int64_t n, const float *T, const float *P,
                               const float *Y, int64_t ldY, float *om, int64_t ldO,
                               cudaStream_t s)
{
    if (!m->have_bf16)
        return set_error(CHEM_EUNSUPPORTED, "split-BF16 path not available for this mechanism");
    if (m->bf16_wide) return launch_source_wide(m, m->bf16, n, T, P, Y, ldY, om, ldO, s);
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
    prm.rct = t->rct;
    prm.fcn = t->fcn;
    prm.bulk_out = (ldO == m->ns && (uintptr_t)om % 16 == 0) ? 1 : 0;
    if ((n + 127) / 128 > 0x7fffffff) return set_error(CHEM_EINVAL, "n_cells too large");
    prm.ntiles = (int)((n + 127) / 128);
    prm.btab = t->btab;
    prm.blob_bytes = (uint32_t)t->blob_bytes;
    prm.invW = t->invW;
    prm.t_mid = (float)m->t_mid;
    prm.lg2R = (float)log2(kR);
    prm.status = t->status;
    // shared memory layout
    auto al = [](size_t x, size_t a) { return (x + a - 1) & ~(a - 1); };
    prm.o_bg = t->o_bg;
    prm.o_b2 = t->o_b2;
    prm.o_e = t->o_e;
    prm.o_qi = t->o_qi;
    prm.o_fq = t->o_fq;
    size_t off = al(prm.blob_bytes, 128);
    const size_t ybytes = (size_t)128 * ldY * 4;
    const size_t fixed = 2 * 512 + al(3 * (size_t)t->nsp * 4, 128) + 2048 + BAR_COUNT * 8 + 64 + 1024;
    const bool aligned = ((uintptr_t)Y % 16 == 0) && ((uintptr_t)T % 16 == 0) && ((uintptr_t)P % 16 == 0);
    prm.stage_y = aligned && (off + ybytes + fixed <= 227 * 1024) ? 1 : 0;
    prm.o_y = (uint32_t)off;
    if (prm.stage_y) off = al(off + ybytes, 128);
    prm.o_t = (uint32_t)off;
    off += 512;
    prm.o_p = (uint32_t)off;
    off += 512;
    prm.o_iw = (uint32_t)off;
    off = al(off + 3 * (size_t)t->nsp * 4, 128);
    prm.o_psum = (uint32_t)off;
    off += 4 * 128 * 4;
    prm.o_bar = (uint32_t)off;
    off += BAR_COUNT * 8 + 64;
    const size_t smem = off + 1024;          // room to align the base to 1024 bytes
    if (smem > 227 * 1024)
        return set_error(CHEM_EUNSUPPORTED, "split-BF16 tables need %zu bytes of shared memory",
                         smem);
    return t->nsp == 32 ? launch_nsp<32>(prm, smem, s, m->device)
                        : launch_nsp<64>(prm, smem, s, m->device);
}

}  // namespace chem
