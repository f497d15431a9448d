// kern_wide.cu -- split-precision source term on tcgen05 tensor cores for mechanisms whose
// tables do not fit in shared memory (more than 53 species, any number of reactions).
//
// The arithmetic is that of kern_bf16.cu (Eqs. 2-11, Sec. 2.4): per tile of 128 cells and
// chunk of RC = 48 reactions, contraction 1 S = A1 . [nu' | nu''] with A1 = [log2 z, log2
// c_tot, normalisation, Arrhenius features] as two FP16 terms, the folded Gibbs layer into
// the reverse half, the rates and falloff factors in an FP32 epilogue, and contraction 2
// omega += q_net . nu^T with q_net as two BF16 terms.  What differs is where the operands
// live, so that the species count can reach ~190:
//   - A1 (128 x NSPW FP16, two terms) is in shared memory, in the core-matrix layout the
//     tensor core reads (each 8-column block of a cell is one 16-byte row of a core matrix);
//     contraction 1 takes A through a shared-memory descriptor;
//   - the stoichiometric tables are streamed from global memory (L2) per chunk through two
//     two-slot rings: [B1 | Gibbs table] of chunk g + 1 is copied as soon as contraction 1
//     of chunk g - 1 has released its slot, B2 likewise after contraction 2;
//   - the third-body sums M / c_tot = 1 + sum_k (eff_k - 1) z_k / sum z (Sec. 2.4) are
//     formed in the epilogue from the listed species (at most kWMaxEff per reaction), with
//     z_k = 2^(log2 z_k) rebuilt from A1's two terms;
//   - T, P and Y are read by the epilogue threads (16-byte loads of three blocks at a time);
//     at the end of a tile omega goes from tensor memory into A1's shared memory (free once
//     every chunk has been evaluated), one odd-strided row per cell, and out to global memory
//     a row per warp instruction, before the next tile's prologue rewrites A1.
// Tensor memory: Gibbs features (16 columns), two S buffers (2 x 96), two q_net buffers
// (2 x 48) and omega (NOUT = 16-padded species count <= 192).
// Roles (480 threads): warp 0 copies the resident tables (share records, third-body lists,
// falloff records); warp 1 issues contraction 1 and keeps its ring filled; warp 14 issues
// contraction 2 and keeps its ring filled; warps 2-13 are three epilogue warpgroups
// (warpgroup g: reactions 16 g .. 16 g + 15 of each chunk; column blocks g, g + 3, ...).
// Every mbarrier wait is bounded (kern_tc_common.cuh): on timeout the kernel records an error
// code in the mechanism's device status word and all roles wind down.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "chem_internal.h"
#include "kern_tc_common.cuh"
#include "tc_ptx.h"

namespace chem {

using namespace tck;

constexpr int kWMaxEff = 8;            // listed third-body efficiencies per reaction
constexpr int kWMaxOut = 192;          // omega columns in tensor memory
constexpr uint32_t kWAG = 0, kWS0 = 32, kWA2 = kWS0 + 4 * RC, kWD2 = kWA2 + 2 * RC;
static_assert(kWD2 + kWMaxOut <= kTmemCols, "tensor memory over budget");

// third-body sum of one multiplier slot: the species whose efficiency differs from 1
struct alignas(16) SlotEff {
    int16_t sp[kWMaxEff];
    float em1[kWMaxEff];
    int32_t n, pad[3];
};

struct WideTables {
    int nspw, nout, nch, rct, qm;
    uint32_t b1c, b2c;                 // bytes per chunk of the two streamed tables
    uint32_t res_bytes, o_qi, o_se, o_fq;
    void *d_blob;
    const unsigned char *b1, *b2, *res;
    const float *invW;
    int *status;
};

struct WideParams {
    const float *T, *P, *Y;
    float *om;
    int64_t n, ldY, ldO;
    int ns, nspw, nout, nch, rct, ntiles;
    const unsigned char *b1, *b2, *res;
    uint32_t b1c, b2c, res_bytes, o_qi, o_se, o_fq;
    const float *invW;
    float t_mid, lg2R;
    int *status;
    // shared-memory layout (offsets from the 1024-aligned base)
    uint32_t o_a1h, o_a1l, o_r1, o_r2, o_res, o_iw, o_psum, o_bar;
};

enum {
    WB_BTAB, WB_A1FULL, WB_D1FULL0, WB_D1FULL1, WB_D1EMPTY0, WB_D1EMPTY1, WB_A2FULL0, WB_A2FULL1,
    WB_A2EMPTY0, WB_A2EMPTY1, WB_B1FULL0, WB_B1FULL1, WB_B1FREE0, WB_B1FREE1, WB_B2FULL0,
    WB_B2FULL1, WB_B2FREE0, WB_B2FREE1, WB_D2FULL, WB_D2EMPTY, WB_XREADY, WB_DRAIN, WB_OSTAGED,
    WB_OCOPIED, WB_COUNT
};

// bulk copy of `bytes` (a multiple of 16) in pieces of at most 16 KiB, completing on `bar`
__device__ __forceinline__ void bulk_copy(uint32_t dst, const unsigned char *src, uint32_t bytes,
                                          uint32_t bar)
{
    tc::mbar_arrive_expect_tx(bar, bytes);
    for (uint32_t off = 0; off < bytes; off += 16384)
        tc::bulk_g2s(dst + off, src + off, min(16384u, bytes - off), bar);
}

__global__ void __launch_bounds__(kThreads, 1) k_source_wide(const WideParams p)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *sm = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
    const uint32_t sbase = tc::smem_u32(sm);
    unsigned char *res = sm + p.o_res;
    const QInfo *qinfo = (const QInfo *)(res + p.o_qi);
    const SlotEff *slot_eff = (const SlotEff *)(res + p.o_se);
    const FallQ *fallq = (const FallQ *)(res + p.o_fq);
    unsigned char *a1h = sm + p.o_a1h, *a1l = sm + p.o_a1l;
    float *iW = (float *)(sm + p.o_iw);           // [nspw] 1 / W_k, zero past the species
    int *ccode = (int *)(iW + p.nspw);            // [nspw] what each column holds
    float *Psum = (float *)(sm + p.o_psum);      // [NQ][128]
    uint64_t *bars = (uint64_t *)(sm + p.o_bar);
    SmemCtl *ctl = (SmemCtl *)(bars + WB_COUNT);
    auto BAR = [&](int i) { return tc::smem_u32(bars + i); };

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int NB = p.nspw / 8;                    // 8-column blocks of A1
    if (tid == 0) {
        constexpr uint32_t E = kEpiWarps;
        const uint32_t cnt[WB_COUNT] = {1, E, 1, 1, E, E, E, E, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1,
                                        1, E, E, 2, E, E};
        for (int i = 0; i < WB_COUNT; ++i) tc::mbar_init(BAR(i), cnt[i]);
        tc::mbar_fence_init();
        ctl->abort = 0;
    }
    if (warp == 1) {
        tc::tmem_alloc(tc::smem_u32(&ctl->tmem_base), kTmemCols);
        tc::tmem_relinquish();
    }
    for (int k = tid; k < p.nspw; k += kThreads) {
        iW[k] = k < p.ns ? p.invW[k] : 0.0f;
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
    // chunks this CTA processes, over all its tiles
    const int ntc = p.ntiles > (int)blockIdx.x ? (p.ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int G = ntc * nch;

    if (warp == 0) {
        // ------------------------------------------------------------- resident tables
        if (lane == 0) {
            bulk_copy(sbase + p.o_res, p.res, p.res_bytes, BAR(WB_BTAB));
            wait_bar(BAR(WB_BTAB), 0, ctl, p.status, 1);
        }
    } else if (warp == 1 || warp == kMma2Warp) {
        // ------------------------------------------------------------- MMA issuers
        if (lane == 0) {
            bool ok = wait_bar(BAR(WB_BTAB), 0, ctl, p.status, 2);
            const uint32_t r1 = sbase + p.o_r1, r2 = sbase + p.o_r2;
            if (warp == 1) {
                // contraction 1 (+ the Gibbs layer) of chunk g into S buffer g & 1; the ring
                // slot of chunk g - 1 is refilled with chunk g + 1 once its MMAs are done
                auto load1 = [&](int g) {
                    bulk_copy(r1 + (uint32_t)(g & 1) * p.b1c, p.b1 + (size_t)(g % nch) * p.b1c,
                              p.b1c, BAR(WB_B1FULL0 + (g & 1)));
                };
                if (G > 0) load1(0);
                int g = 0;
                const uint32_t a_h = sbase + p.o_a1h, a_l = sbase + p.o_a1l;
                for (int it = 0; ok && it < ntc; ++it) {
                    if (!(ok = wait_bar(BAR(WB_A1FULL), it & 1, ctl, p.status, 2))) break;
                    for (int c = 0; c < nch; ++c, ++g) {
                        const int b = g & 1;
                        if (!(ok = wait_bar(BAR(WB_D1EMPTY0 + b), ((g >> 1) & 1) ^ 1, ctl, p.status, 2)))
                            break;
                        if (!(ok = wait_bar(BAR(WB_B1FULL0 + b), (g >> 1) & 1, ctl, p.status, 2))) break;
                        tc::fence_after();
                        const int rcc = c == nch - 1 ? p.rct : RC;
                        const uint32_t d = tmem + kWS0 + (uint32_t)b * (2 * RC);
                        const uint32_t id1 = tc::idesc_f16_f32(128, 2 * rcc);
                        const uint32_t bc = r1 + (uint32_t)b * p.b1c;
                        for (int s = 0; s < 2; ++s)
                            for (int kk = 0; kk < NB / 2; ++kk)
                                tc::mma_ss(d, tc::sdesc_noswz((s ? a_l : a_h) + kk * 256, 128, NB * 128),
                                           tc::sdesc_noswz(bc + kk * 256, 128, NB * 128), id1,
                                           (s | kk) != 0);
                        const uint32_t idg = tc::idesc_f16_f32(128, rcc);
                        const uint32_t gc = bc + (uint32_t)(2 * RC * p.nspw * 2);
#pragma unroll
                        for (int s = 0; s < 2; ++s)
#pragma unroll
                            for (int tt = 0; tt < 2 - s; ++tt)
                                tc::mma_ts(d + rcc, tmem + kWAG + s * 8,
                                           tc::sdesc_noswz(gc + tt * 256, 128, (kGibK / 8) * 128),
                                           idg, 1);
                        tc::commit(BAR(WB_D1FULL0 + b));
                        tc::commit(BAR(WB_B1FREE0 + b));
                        if (g + 1 < G) {
                            // slot (g + 1) & 1 was last read by chunk g - 1
                            if (g >= 1 && !(ok = wait_bar(BAR(WB_B1FREE0 + ((g + 1) & 1)),
                                                          ((g - 1) >> 1) & 1, ctl, p.status, 2)))
                                break;
                            load1(g + 1);
                        }
                    }
                }
                // the ring's last copy has landed before the CTA can exit
                if (G > 0) wait_bar(BAR(WB_B1FULL0 + ((G - 1) & 1)), ((G - 1) >> 1) & 1, ctl, p.status, 2);
            } else {
                // contraction 2 of each chunk in chunk order; the first of a tile once the
                // tile before's omega has been read out (D2EMPTY)
                auto load2 = [&](int g) {
                    bulk_copy(r2 + (uint32_t)(g & 1) * p.b2c, p.b2 + (size_t)(g % nch) * p.b2c,
                              p.b2c, BAR(WB_B2FULL0 + (g & 1)));
                };
                if (G > 0) load2(0);
                const uint32_t id2 = tc::idesc_bf16_f32(128, p.nout);
                int g = 0;
                for (int it = 0; ok && it < ntc; ++it) {
                    if (it > 0 && !(ok = wait_bar(BAR(WB_D2EMPTY), (it - 1) & 1, ctl, p.status, 2)))
                        break;
                    for (int c = 0; c < nch; ++c, ++g) {
                        const int ab = g & 1;
                        if (!(ok = wait_bar(BAR(WB_A2FULL0 + ab), (g >> 1) & 1, ctl, p.status, 2))) break;
                        if (!(ok = wait_bar(BAR(WB_B2FULL0 + ab), (g >> 1) & 1, ctl, p.status, 2))) break;
                        tc::fence_after();
                        const int rcc = c == nch - 1 ? p.rct : RC;
                        const uint32_t bc = r2 + (uint32_t)ab * p.b2c;
                        const uint32_t a2 = tmem + kWA2 + (uint32_t)ab * RC;
                        for (int s = 0; s < 2; ++s)
                            for (int kk = 0; kk < rcc / 16; ++kk)
                                tc::mma_ts(tmem + kWD2, a2 + s * (RC / 2) + kk * 8,
                                           tc::sdesc_noswz(bc + kk * 256, 128, (rcc / 8) * 128), id2,
                                           (c | s | kk) != 0);
                        tc::commit(BAR(WB_A2EMPTY0 + ab));
                        tc::commit(BAR(WB_B2FREE0 + ab));
                        if (g + 1 < G) {
                            if (g >= 1 && !(ok = wait_bar(BAR(WB_B2FREE0 + ((g + 1) & 1)),
                                                          ((g - 1) >> 1) & 1, ctl, p.status, 2)))
                                break;
                            load2(g + 1);
                        }
                    }
                    if (ok) tc::commit(BAR(WB_D2FULL));
                }
                if (G > 0) wait_bar(BAR(WB_B2FULL0 + ((G - 1) & 1)), ((G - 1) >> 1) & 1, ctl, p.status, 2);
            }
            tc::commit(BAR(WB_DRAIN));
            wait_bar(BAR(WB_DRAIN), 0, ctl, p.status, 2);
        }
    } else if (warp < kMma2Warp) {
        // ------------------------------------------------------------- epilogue
        const int ew = warp - kEpiWarp0;
        const int g = ew >> 2;
        const int q = warp & 3;
        const int row = q * 32 + lane;
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        const int ns = p.ns;
        bool ok = wait_bar(BAR(WB_BTAB), 0, ctl, p.status, 3);
        // byte offset of (this cell, 8-column block blk) in A1's core-matrix layout
        const uint32_t rowoff = (uint32_t)(row >> 3) * (uint32_t)NB * 128u + (uint32_t)(row & 7) * 16u;
        auto prologue = [&](int t, int itp, CellF &cf) -> bool {
            const int64_t ci = (int64_t)t * 128 + row;
            float Tc = 1000.0f, Pc = 1.0e6f;
            const float *yrow = nullptr;
            if (ci < n) {
                Tc = __ldg(p.T + ci);
                Pc = __ldg(p.P + ci);
                yrow = p.Y + ci * p.ldY;
            }
            cf.lg2T = log2f(Tc);
            cf.invT = 1.0f / Tc;
            cf.itau = 1000.0f / Tc;
            cf.T = Tc;
            cf.lgct = log2f(Pc) - p.lg2R - cf.lg2T;
            float psum = 0.0f;
            // rows that start on a 16-byte boundary are read 16 bytes at a time
            const bool yvec = yrow && (((uintptr_t)yrow) & 15) == 0;
            // the Y values of three of this thread's blocks at a time, so that their loads
            // are in flight together
            constexpr int kBMax = (kWMaxOut + 2 + kArrRows + 15) / 16 * 2 / NQ + 1;
            for (int b0 = 0; b0 < kBMax; b0 += 3) {
                float yv[3][8];
#pragma unroll
                for (int bi = 0; bi < 3; ++bi) {
                    const int blk = g + NQ * (b0 + bi);
                    if (yvec && 8 * blk + 8 <= ns) {
                        // a block inside the row: two 16-byte loads
                        const float4 v0 = __ldg((const float4 *)(yrow + 8 * blk));
                        const float4 v1 = __ldg((const float4 *)(yrow + 8 * blk + 4));
                        yv[bi][0] = v0.x; yv[bi][1] = v0.y; yv[bi][2] = v0.z; yv[bi][3] = v0.w;
                        yv[bi][4] = v1.x; yv[bi][5] = v1.y; yv[bi][6] = v1.z; yv[bi][7] = v1.w;
                    } else {
#pragma unroll
                        for (int e = 0; e < 8; ++e)
                            yv[bi][e] = (yrow && blk < NB) ? __ldg(yrow + min(8 * blk + e, ns - 1)) : 0.0f;
                    }
                }
#pragma unroll
                for (int bi = 0; bi < 3; ++bi) {
                    const int blk = g + NQ * (b0 + bi);
                    if (blk < NB) {
                        float lx[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const int k = 8 * blk + e;
                            const float z = fmaxf(yv[bi][e], 0.0f) * iW[k];
                            psum += z;
                            const float lz = fmaxf(tc::lg2(z), kLog2Floor);
                            const int cc = ccode[k];
                            lx[e] = cc == kColSpecies ? lz : cc == kColLgct ? cf.lgct
                                  : cc == kColOne ? 1.0f : cc == kColLg2T ? cf.lg2T
                                  : cc == kColItau ? cf.itau : 0.0f;
                        }
                        uint4 wh, wl;
                        split2h(lx[0], lx[1], wh.x, wl.x);
                        split2h(lx[2], lx[3], wh.y, wl.y);
                        split2h(lx[4], lx[5], wh.z, wl.z);
                        split2h(lx[6], lx[7], wh.w, wl.w);
                        *(uint4 *)(a1h + rowoff + (uint32_t)blk * 128u) = wh;
                        *(uint4 *)(a1l + rowoff + (uint32_t)blk * 128u) = wl;
                    }
                }
            }
            Psum[g * 128 + row] = psum;
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(BAR(WB_XREADY));
            tc::fence_after();
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
                const uint32_t ag = tmem + lane_off + kWAG;
                tc::tmem_st8(ag + 0, gh);
                tc::tmem_st8(ag + 8, gl);
            }
            if (!wait_bar(BAR(WB_XREADY), itp & 1, ctl, p.status, 3)) return false;
            float sum = 0.0f;
#pragma unroll
            for (int gg = 0; gg < NQ; ++gg) sum += Psum[gg * 128 + row];
            cf.inv_sum = sum > 0.0f ? 1.0f / sum : 0.0f;
            {
                // the normalisation column ns + 1 (both terms), in its block's 16-byte row
                const int kn = ns + 1;
                if ((kn >> 3) % NQ == g) {
                    const float vn = sum > 0.0f ? cf.lgct - log2f(sum) : 0.0f;
                    uint32_t h, l;
                    split2h(vn, 0.0f, h, l);
                    const uint32_t o = rowoff + (uint32_t)(kn >> 3) * 128u + (uint32_t)(kn & 7) * 2u;
                    *(uint16_t *)(a1h + o) = (uint16_t)(h & 0xFFFFu);
                    *(uint16_t *)(a1l + o) = (uint16_t)(l & 0xFFFFu);
                }
            }
            tc::fence_proxy_async_smem();             // A1 visible to the tensor core
            tc::tmem_wait_st();
            tc::fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(BAR(WB_A1FULL));
            return true;
        };
        // z_k of this cell rebuilt from A1's two terms of log2 z_k
        auto z_of = [&](int k) -> float {
            const uint32_t o = rowoff + (uint32_t)(k >> 3) * 128u + (uint32_t)(k & 7) * 2u;
            const __half h = *(const __half *)(a1h + o), l = *(const __half *)(a1l + o);
            return tc::ex2(__half2float(h) + __half2float(l));
        };
        CellF cf, cfn;
        int it = 0;
        uint32_t u = 0;
        if ((int)blockIdx.x < p.ntiles) ok = ok && prologue(blockIdx.x, 0, cf);
        for (int t = blockIdx.x; ok && t < p.ntiles; t += gridDim.x, ++it) {
            const int t_next = t + gridDim.x;
            const bool has_next = t_next < p.ntiles;
            uint32_t sf[RH], sr[RH];
            auto load_s = [&](int c, uint32_t uu) -> bool {
                const int b = (int)(uu & 1);
                if (!wait_bar(BAR(WB_D1FULL0 + b), (uu >> 1) & 1, ctl, p.status, 3)) return false;
                tc::fence_after();
                const int rcc = c == nch - 1 ? p.rct : RC;
                if (g * RH < rcc) {
                    const uint32_t d1 = tmem + lane_off + kWS0 + (uint32_t)b * (2 * RC) + g * RH;
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
                if (lane == 0) tc::mbar_arrive(BAR(WB_D1EMPTY0 + (int)(uu & 1)));
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
                        // third-body / falloff slots 0..7 of a multiplier share: M / c_tot =
                        // 1 + sum over the listed species of (eff - 1) z_k / sum z
                        float s8[8], fac[4], mul[4];
                        const SlotEff *se = slot_eff + 8 * qi.rank;
#pragma unroll
                        for (int r = 0; r < 8; ++r) {
                            float acc = 0.0f;
                            const int ne = se[r].n;
                            for (int i = 0; i < ne; ++i) acc = fmaf(se[r].em1[i], z_of(se[r].sp[i]), acc);
                            s8[r] = fmaf(acc, cf.inv_sum, 1.0f);
                        }
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
                if (c + 1 < nch && !(ok = load_s(c + 1, u + 1))) break;
                const int ab = (int)(u & 1);
                if (!(ok = wait_bar(BAR(WB_A2EMPTY0 + ab), ((u >> 1) & 1) ^ 1, ctl, p.status, 3))) break;
                tc::fence_after();
                if (active) {
                    const uint32_t a2 = tmem + lane_off + kWA2 + (uint32_t)ab * RC + g * (RH / 2);
                    tc::tmem_st8(a2, hw);
                    tc::tmem_st8(a2 + RC / 2, lw);
                    tc::tmem_wait_st();
                }
                tc::fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(BAR(WB_A2FULL0 + ab));
                if (c == nch - 1) {
                    // every warp has finished reading A1 (third-body z) for this tile: omega
                    // goes out through A1's shared memory (one padded row per cell, copied
                    // to global memory a row per warp instruction), then the next tile's
                    // prologue rewrites A1
                    if (!(ok = wait_bar(BAR(WB_A2FULL0 + ab), (u >> 1) & 1, ctl, p.status, 3))) break;
                    if (!(ok = wait_bar(BAR(WB_D2FULL), it & 1, ctl, p.status, 3))) break;
                    tc::fence_after();
                    float *Ws = (float *)a1h;
                    const int ldw = ns | 1;           // odd: conflict-free columns and rows
                    for (int blk = g; blk < p.nout / 8; blk += NQ) {
                        uint32_t w[8];
                        tc::tmem_ld8(tmem + lane_off + kWD2 + 8 * blk, w);
#pragma unroll
                        for (int e = 0; e < 8; ++e)
                            if (8 * blk + e < ns) Ws[row * ldw + 8 * blk + e] = __uint_as_float(w[e]);
                    }
                    tc::fence_before();
                    __syncwarp();
                    if (lane == 0) {
                        tc::mbar_arrive(BAR(WB_D2EMPTY));
                        tc::mbar_arrive(BAR(WB_OSTAGED));
                    }
                    if (!(ok = wait_bar(BAR(WB_OSTAGED), it & 1, ctl, p.status, 3))) break;
                    const int64_t i0 = (int64_t)t * 128;
                    for (int r = warp - kEpiWarp0; r < 128; r += kEpiWarps) {
                        if (i0 + r >= n) break;
                        float *orow = p.om + (i0 + r) * p.ldO;
                        for (int k = lane; k < ns; k += 32) orow[k] = Ws[r * ldw + k];
                    }
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(BAR(WB_OCOPIED));
                    if (!(ok = wait_bar(BAR(WB_OCOPIED), it & 1, ctl, p.status, 3))) break;
                    if (has_next && !(ok = prologue(t_next, it + 1, cfn))) break;
                }
                if (c + 1 < nch) release_s(c + 1, u + 1);
            }
            if (!ok) break;
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
// host side
// ---------------------------------------------------------------------------------------

// Maximum species count of this path (tensor-memory omega columns).
int wide_max_species() { return kWMaxOut; }

chem_status wide_build_tables(chem_mech *m, const chem_mech_desc *d, void **out)
{
    const int ns = d->n_species, nr = d->n_reactions;
    const int nspw = ((ns + 2 + kArrRows + 15) / 16) * 16;
    const int nout = ((ns + 15) / 16) * 16;
    if (nout > kWMaxOut)
        return set_error(CHEM_EUNSUPPORTED, "split-BF16 path supports up to %d species", kWMaxOut);
    const int kf0 = ns + 2;
    const int nrp = ((nr + 15) / 16) * 16;
    const int nch = (nrp + RC - 1) / RC;
    const int rct = nrp - (nch - 1) * RC;
    std::vector<int> plain, fall, tbr;
    for (int j = 0; j < nr; ++j)
        (d->kind[j] == 0 ? plain : d->kind[j] == CHEM_RXN_THIRD_BODY ? tbr : fall).push_back(j);
    const int nspec = (int)(fall.size() + tbr.size());
    int qm = 0;
    if (nspec) qm = std::max((nspec + 7) / 8, ((int)fall.size() + 3) / 4);
    std::vector<int> shares;                   // multiplier shares from the end, chunk 0 last
    for (int c = nch - 1; c >= 1; --c)
        for (int gq = (c == nch - 1 ? rct / RH : NQ) - 1; gq >= 0; --gq) shares.push_back(c * NQ + gq);
    for (int gq = (nch == 1 ? rct / RH : NQ) - 1; gq >= 0; --gq) shares.push_back(gq);
    if (qm > (int)shares.size())
        return set_error(CHEM_EUNSUPPORTED,
                         "split-BF16 path: %d third-body / falloff reactions (%d falloff) exceed "
                         "the multiplier slots", nspec, (int)fall.size());
    std::vector<QInfo> qinfo((size_t)nch * NQ);
    for (auto &x : qinfo) x = QInfo{-1, 0, 0, 0};
    std::vector<int> qsel(shares.begin(), shares.begin() + qm);
    std::sort(qsel.begin(), qsel.end());
    for (int r = 0; r < qm; ++r) qinfo[qsel[r]].rank = (int8_t)r;
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
            if (fill[r] >= 8) return set_error(CHEM_EUNSUPPORTED, "split-BF16 path: multiplier slots");
            order[slot_of(qsel[r], fill[r]++)] = tbr[i];
        }
        size_t pi = 0;
        for (int c = 0; c < nch && pi < plain.size(); ++c)
            for (int r = 0; r < (c == nch - 1 ? rct : RC) && pi < plain.size(); ++r)
                if (order[(size_t)c * RC + r] < 0) order[(size_t)c * RC + r] = plain[pi++];
        if (pi != plain.size()) return set_error(CHEM_EUNSUPPORTED, "split-BF16 path: slot layout");
    }
    // streamed tables, one block per chunk: [B1: 2 RC rows x nspw | BG: RC rows x 32] FP16
    // and B2: nout rows x RC BF16 (core-matrix order, K-major; the last chunk uses its rows)
    const uint32_t b1c = (uint32_t)(2 * RC * nspw * 2 + RC * kGibK * 2);
    const uint32_t b2c = (uint32_t)(nout * RC * 2);
    std::vector<uint16_t> b1((size_t)nch * b1c / 2, 0), b2((size_t)nch * b2c / 2, 0);
    auto b1_at = [&](int c, int r, int k) -> uint16_t & {
        return b1[(size_t)c * b1c / 2 + ((r / 8) * (nspw / 8) + k / 8) * 64 + (r % 8) * 8 + k % 8];
    };
    auto bg_at = [&](int c, int r, int k) -> uint16_t & {
        return b1[(size_t)c * b1c / 2 + (size_t)2 * RC * nspw + ((r / 8) * (kGibK / 8) + k / 8) * 64 +
                  (r % 8) * 8 + k % 8];
    };
    auto b2_at = [&](int c, int rcc, int nrow, int r) -> uint16_t & {
        return b2[(size_t)c * b2c / 2 + ((nrow / 8) * (rcc / 8) + r / 8) * 64 + (nrow % 8) * 8 + r % 8];
    };
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
    std::vector<SlotEff> se((size_t)std::max(qm, 1) * 8);
    memset(se.data(), 0, se.size() * sizeof(SlotEff));
    std::vector<int> qrank((size_t)nch * NQ, -1);
    for (int r = 0; r < qm; ++r) qrank[qsel[r]] = r;
    uint16_t dead[3];
    f16_split<3>(kDead, dead);
    for (int c = 0; c < nch; ++c) {
        const int rcc = c == nch - 1 ? rct : RC;
        for (int r = 0; r < rcc; ++r) {
            const int j = order[(size_t)c * RC + r];
            if (j < 0) {
                for (int i = 0; i < 3; ++i) b1_at(c, r, kf0 + i) = b1_at(c, rcc + r, kf0 + i) = dead[i];
                continue;
            }
            const int kind = d->kind[j];
            const double *ar = d->arrh + (size_t)j * 3;
            int ordf = 0, ordr = 0;
            for (int k = 0; k < ns; ++k) {
                const int f = d->nu_f[(size_t)j * ns + k], pr = d->nu_r[(size_t)j * ns + k];
                ordf += f;
                ordr += pr;
                b1_at(c, r, k) = f16_of_int(f);
                b1_at(c, rcc + r, k) = f16_of_int(pr);
                b2_at(c, rcc, k, r) = bf16_of_int(pr - f);
            }
            const int tbx = kind == CHEM_RXN_THIRD_BODY ? 1 : 0;
            b1_at(c, r, ns) = f16_of_int(tbx);
            b1_at(c, rcc + r, ns) = f16_of_int(tbx);
            b1_at(c, r, ns + 1) = f16_of_int(ordf);
            b1_at(c, rcc + r, ns + 1) = f16_of_int(ordr);
            const double co[3] = {ar[0] * kLog2e, ar[1], -ar[2] * kLog2e * 1e-3};
            for (int f = 0; f < 3; ++f) {
                uint16_t t3[3];
                f16_split<3>(co[f], t3);
                for (int i = 0; i < 3; ++i) {
                    b1_at(c, r, kf0 + 3 * f + i) = t3[i];
                    if (d->reversible[j]) b1_at(c, rcc + r, kf0 + 3 * f + i) = t3[i];
                }
            }
            if (!d->reversible[j]) {
                for (int i = 0; i < 3; ++i) b1_at(c, rcc + r, kf0 + i) = dead[i];
            } else {
                for (int rg = 0; rg < 2; ++rg)
                    for (int qq = 0; qq < 7; ++qq) {
                        double cj = 0.0;
                        for (int k = 0; k < ns; ++k) {
                            const int nu = d->nu_r[(size_t)j * ns + k] - d->nu_f[(size_t)j * ns + k];
                            if (nu) cj += nu * gsp[(size_t)k * 14 + rg * 7 + qq];
                        }
                        uint16_t t2[2];
                        f16_split<2>(cj, t2);
                        for (int i = 0; i < 2; ++i) bg_at(c, r, 16 * i + 7 * rg + qq) = t2[i];
                    }
            }
            if (kind == 0) continue;
            const int qq = c * NQ + r / RH, pos = r % RH;
            const int rk = qrank[qq];
            if (rk < 0 || pos >= 8 || (kind != CHEM_RXN_THIRD_BODY && pos >= 4))
                return set_error(CHEM_EUNSUPPORTED, "split-BF16 path: multiplier slot layout");
            SlotEff &E = se[(size_t)8 * rk + pos];
            for (int k = 0; k < ns; ++k) {
                const double e = (d->eff ? d->eff[(size_t)j * ns + k] : 1.0) - 1.0;
                if (e == 0.0) continue;
                if (E.n >= kWMaxEff)
                    return set_error(CHEM_EUNSUPPORTED,
                                     "split-BF16 path (large mechanisms): reaction %d lists more "
                                     "than %d third-body efficiencies", j, kWMaxEff);
                E.sp[E.n] = (int16_t)k;
                E.em1[E.n] = (float)e;
                ++E.n;
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
    // device blob: B1 chunks | B2 chunks | resident block (share records | slot lists |
    // falloff) | 1/W | status word
    auto a256 = [](size_t x) { return (x + 255) & ~(size_t)255; };
    auto a16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
    const size_t ob1 = 0, ob2 = a256(b1.size() * 2), ores = a256(ob2 + b2.size() * 2);
    const size_t oqi = 0, ose = a16(oqi + qinfo.size() * sizeof(QInfo)),
                 ofq = a16(ose + se.size() * sizeof(SlotEff)),
                 res_bytes = a16(ofq + fq.size() * sizeof(FallQ));
    const size_t oiw = a256(ores + res_bytes), ost = a256(oiw + invW.size() * 4), total = a256(ost + 16);
    std::vector<unsigned char> h(total, 0);
    memcpy(h.data() + ob1, b1.data(), b1.size() * 2);
    memcpy(h.data() + ob2, b2.data(), b2.size() * 2);
    memcpy(h.data() + ores + oqi, qinfo.data(), qinfo.size() * sizeof(QInfo));
    memcpy(h.data() + ores + ose, se.data(), se.size() * sizeof(SlotEff));
    memcpy(h.data() + ores + ofq, fq.data(), fq.size() * sizeof(FallQ));
    memcpy(h.data() + oiw, invW.data(), invW.size() * 4);
    WideTables *t = new (std::nothrow) WideTables();
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
    t->nspw = nspw;
    t->nout = nout;
    t->nch = nch;
    t->rct = rct;
    t->qm = qm;
    t->b1c = b1c;
    t->b2c = b2c;
    t->res_bytes = (uint32_t)res_bytes;
    t->o_qi = (uint32_t)oqi;
    t->o_se = (uint32_t)ose;
    t->o_fq = (uint32_t)ofq;
    t->b1 = base + ob1;
    t->b2 = base + ob2;
    t->res = base + ores;
    t->invW = (const float *)(base + oiw);
    t->status = (int *)(base + ost);
    m->device_bytes += total;
    *out = t;
    return CHEM_OK;
}

void wide_free_tables(void *p)
{
    WideTables *t = (WideTables *)p;
    if (!t) return;
    cudaFree(t->d_blob);
    delete t;
}

int *wide_status_word(const void *p) { return ((const WideTables *)p)->status; }

// Shared memory the launch needs (0 if it does not fit).
static size_t wide_smem(const WideTables *t, WideParams *prm)
{
    auto al = [](size_t x, size_t a) { return (x + a - 1) & ~(a - 1); };
    size_t off = 0;
    prm->o_a1h = (uint32_t)off;
    off = al(off + (size_t)128 * t->nspw * 2, 1024);
    prm->o_a1l = (uint32_t)off;
    off = al(off + (size_t)128 * t->nspw * 2, 1024);
    prm->o_r1 = (uint32_t)off;
    off = al(off + 2 * (size_t)t->b1c, 1024);
    prm->o_r2 = (uint32_t)off;
    off = al(off + 2 * (size_t)t->b2c, 1024);
    prm->o_res = (uint32_t)off;
    off = al(off + t->res_bytes, 128);
    prm->o_iw = (uint32_t)off;
    off = al(off + 2 * (size_t)t->nspw * 4, 128);
    prm->o_psum = (uint32_t)off;
    off += NQ * 128 * 4;
    prm->o_bar = (uint32_t)off;
    off += WB_COUNT * 8 + 64;
    return off + 1024;
}

chem_status wide_check(const void *p)
{
    const WideTables *t = (const WideTables *)p;
    WideParams prm;
    const size_t smem = wide_smem(t, &prm);
    if (smem > 227 * 1024)
        return set_error(CHEM_EUNSUPPORTED,
                         "split-BF16 path: operands and table rings need %zu bytes of shared "
                         "memory", smem);
    return CHEM_OK;
}

chem_status launch_source_wide(const chem_mech *m, const void *tables, int64_t n, const float *T,
                               const float *P, const float *Y, int64_t ldY, float *om, int64_t ldO,
                               cudaStream_t s)
{
    const WideTables *t = (const WideTables *)tables;
    WideParams prm;
    memset(&prm, 0, sizeof prm);
    const size_t smem = wide_smem(t, &prm);
    if (smem > 227 * 1024)
        return set_error(CHEM_EUNSUPPORTED, "split-BF16 path needs %zu bytes of shared memory", smem);
    if ((n + 127) / 128 > 0x7fffffff) return set_error(CHEM_EINVAL, "n_cells too large");
    prm.T = T;
    prm.P = P;
    prm.Y = Y;
    prm.om = om;
    prm.n = n;
    prm.ldY = ldY;
    prm.ldO = ldO;
    prm.ns = m->ns;
    prm.nspw = t->nspw;
    prm.nout = t->nout;
    prm.nch = t->nch;
    prm.rct = t->rct;
    prm.ntiles = (int)((n + 127) / 128);
    prm.b1 = t->b1;
    prm.b2 = t->b2;
    prm.res = t->res;
    prm.b1c = t->b1c;
    prm.b2c = t->b2c;
    prm.res_bytes = t->res_bytes;
    prm.o_qi = t->o_qi;
    prm.o_se = t->o_se;
    prm.o_fq = t->o_fq;
    prm.invW = t->invW;
    prm.t_mid = (float)m->t_mid;
    prm.lg2R = (float)log2(kR);
    prm.status = t->status;
    static SmemOptIn opt;
    const int grid = std::min(prm.ntiles, sm_limit(sm_count(m->device)));
    chem_status st = launch_opted(opt, (const void *)k_source_wide, 227 * 1024, "split-BF16 (wide)",
                                  [&] { k_source_wide<<<grid, kThreads, smem, s>>>(prm); });
    if (st == CHEM_OK) g_launches.fetch_add(1);
    return st;
}

}  // namespace chem
