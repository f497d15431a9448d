// kern_tc_common.cuh -- pieces shared by the split-precision tensor-core source-term kernels
// (kern_bf16.cu: mechanism tables resident in shared memory; kern_wide.cu: tables streamed
// from L2 for large mechanisms): chunk geometry, falloff layer, operand splits, bounded
// mbarrier waits, and the host-side 16-bit encodings of the tables.
#pragma once

#include <cuda_fp16.h>
#include <string.h>

#include "chem_internal.h"
#include "tc_ptx.h"

namespace chem {
namespace tck {

constexpr int RC = 48;                 // reactions per chunk
constexpr int RH = 16;                 // reactions per warpgroup and chunk
constexpr int NQ = RC / RH;            // epilogue warpgroups (chunk shares)
constexpr int kEpiWarp0 = 2;           // first epilogue warp
constexpr int kEpiWarps = 4 * NQ;
constexpr int kMma2Warp = kEpiWarp0 + kEpiWarps;   // issues contractions 0 and 2
constexpr int kThreads = 32 * (kMma2Warp + 1);
constexpr uint32_t kTmemCols = 512;
constexpr float kLog2Floor = -1000.0f; // log2 X of an absent species: 2^x underflows to 0
constexpr float kDead = -1.0e4f;       // log2 of a rate constant that is zero
constexpr int kArrRows = 9;            // K rows of the Arrhenius layer: 3 features x 3 terms
constexpr int kGibK = 32;              // K of the Gibbs contraction: 2 coefficient terms x 16
// what a contraction-1 column holds: log2 z_k, log2 c_tot, the normalisation, the Arrhenius
// features 1, log2 T, 1000/T, or nothing
enum { kColSpecies, kColLgct, kColNorm, kColOne, kColLg2T, kColItau, kColZero };

// Falloff layer of slot 0..3 of a multiplier share (Sec. 2.4); neutral records (kf.w = 0)
// leave the third-body factor M / c_tot.
struct alignas(16) FallQ {
    float4 kf;         // log2 k_inf = x + y log2 T + z / T; w = 1 for a falloff reaction
    float4 k0;         // log2 k0 = x + y log2 T + z / T
    float4 troe;       // 1 - alpha, alpha, log2(e)/T***, log2(e)/T* (Lindemann: 1, 0, 0, 0)
    float4 t2;         // x = log2(e) T** (absent: 1e30, the term underflows to zero)
};

// per chunk share (chunk, warpgroup): its rank among the multiplier shares (-1: none) and
// how many of its slots 0..3 hold falloff reactions
struct QInfo {
    int8_t rank, nfall, pad0, pad1;
};

struct SmemCtl {
    uint32_t tmem_base;
    volatile int abort;
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

// Per-cell features kept in registers by every epilogue thread.
struct CellF {
    float lg2T, invT, itau, T, lgct, inv_sum;
};

// Factors of slots 0..3 of a multiplier share from s = M / c_tot (Sec. 2.4): a falloff
// slot (u < nfall) gets fac = log2(Pr / (1 + Pr) F) (F = 1 for Lindemann, the Troe form
// otherwise), added to both exponents, and mul = 1; the others keep fac = 0, mul = s.
__device__ __forceinline__ void falloff4(const FallQ *F, const float (&s)[8], const CellF &c,
                                         int nfall, float (&fac)[4], float (&mul)[4])
{
    constexpr float kLog10_2 = 0.30102999566398120f;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        fac[u] = 0.0f;
        mul[u] = s[u];
        if (u < nfall) {                                          // warp-uniform
            const float4 kf = F[u].kf, k0 = F[u].k0, tr = F[u].troe;
            const float t2 = F[u].t2.x;
            const float lkf = fmaf(kf.z, c.invT, fmaf(kf.y, c.lg2T, kf.x));
            const float lk0 = fmaf(k0.z, c.invT, fmaf(k0.y, c.lg2T, k0.x));
            const float lpr = lk0 - lkf + c.lgct + tc::lg2(fmaxf(s[u], 1e-30f));   // log2 Pr
            float f = -tc::lg2(1.0f + tc::ex2(-lpr));                 // log2(Pr / (1 + Pr))
            const float fc = tr.x * tc::ex2(-c.T * tr.z) + tr.y * tc::ex2(-c.T * tr.w) +
                             tc::ex2(-t2 * c.invT);
            const float lfc = tc::lg2(fc);                            // log2 F_cent
            const float l10 = lfc * kLog10_2;
            const float cc = -0.4f - 0.67f * l10, nn = 0.75f - 1.27f * l10;
            const float x = fmaf(lpr, kLog10_2, cc);
            const float dd = fmaf(-0.14f, x, nn);
            // log2 F = log2 F_cent / (1 + (x / dd)^2)
            f += lfc * __fdividef(dd * dd, fmaf(dd, dd, x * x));
            fac[u] = f;
            mul[u] = 1.0f;
        }
    }
}

// two values -> two packed FP16x2 words (hi, lo terms; value a in the low halves)
__device__ __forceinline__ void split2h(float a, float b, uint32_t &h, uint32_t &l)
{
    h = tc::pack_f16x2(a, b);
    float ha, hb;
    tc::unpack_f16x2(h, ha, hb);
    l = tc::pack_f16x2(a - ha, b - hb);
}

// two values -> two packed BF16x2 words (hi, lo terms; value a in the low halves)
__device__ __forceinline__ void split2x2(float a, float b, uint32_t &h, uint32_t &l)
{
    h = tc::pack_bf16x2(a, b);
    l = tc::pack_bf16x2(a - __uint_as_float(h << 16), b - __uint_as_float(h & 0xFFFF0000u));
}

// ---- host side: 16-bit encodings of the tables

inline uint16_t bf16_of_int(int v)
{
    float f = (float)v;
    uint32_t u;
    memcpy(&u, &f, 4);
    return (uint16_t)(u >> 16);              // exact for |v| <= 256
}

inline uint16_t bf16_rn(float f)
{
    uint32_t u;
    memcpy(&u, &f, 4);
    return (uint16_t)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);   // nearest, ties to even
}

inline double f_of_bf16(uint16_t h)
{
    const uint32_t u = (uint32_t)h << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

inline uint16_t f16_rn(double x)
{
    const __half_raw r = __float2half_rn((float)x);
    return r.x;
}

inline double f_of_f16(uint16_t u)
{
    __half_raw r;
    r.x = u;
    return (double)__half2float(__half(r));
}

inline uint16_t f16_of_int(int v) { return f16_rn((double)v); }   // exact for |v| <= 2048

// x = t[0] + t[1] + ..., each term the nearest FP16 of the remaining residual
template <int N>
inline void f16_split(double x, uint16_t (&t)[N])
{
    for (int i = 0; i < N; ++i) {
        t[i] = f16_rn(x);
        x -= f_of_f16(t[i]);
    }
}

inline int sm_count(int dev)
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


}  // namespace tck
}  // namespace chem
