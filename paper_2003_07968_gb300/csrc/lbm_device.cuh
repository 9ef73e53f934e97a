// lbm_device.cuh -- device-side data layout and per-site arithmetic of the
// D2Q9 pseudopotential step (arXiv 2003.07968) for sm_103a.
//
// Layout in HBM (per lattice, per population buffer):
//   nine SoA planes, one per velocity c_i (Eq. VelocitySet order), each a
//   pitched 2-D array with a ghost frame: rows [-GY, ny+GY), columns
//   [-gx, pitch-gx).  Ghost sites within GW of the interior hold periodic
//   images, written by the same kernel that writes the interior site, so
//   readers never wrap indices.  Two population buffers (A/B) alternate
//   between steps; a float psi plane with the same ghost frame sits beside.
//   The buffers hold POST-collision, PRE-streaming populations f*; a step
//   pulls f_i(x) = f*_i(x - c_i) (streaming of Eq. TLBE in pull form).
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace pplbm {

constexpr int GW = 2;  // depth of the periodic images kept around the interior
constexpr int GY = 2;  // ghost rows above and below

// D2Q9 velocity set, Eq. (VelocitySet); weights from the text after Eq. (SEDF).
__device__ __constant__ static const int kCx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__device__ __constant__ static const int kCy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

template <int I> struct Vel;
template <> struct Vel<0> { static constexpr int x = 0, y = 0; static constexpr float w = 4.f / 9.f; };
template <> struct Vel<1> { static constexpr int x = 1, y = 0; static constexpr float w = 1.f / 9.f; };
template <> struct Vel<2> { static constexpr int x = 0, y = 1; static constexpr float w = 1.f / 9.f; };
template <> struct Vel<3> { static constexpr int x = -1, y = 0; static constexpr float w = 1.f / 9.f; };
template <> struct Vel<4> { static constexpr int x = 0, y = -1; static constexpr float w = 1.f / 9.f; };
template <> struct Vel<5> { static constexpr int x = 1, y = 1; static constexpr float w = 1.f / 36.f; };
template <> struct Vel<6> { static constexpr int x = -1, y = 1; static constexpr float w = 1.f / 36.f; };
template <> struct Vel<7> { static constexpr int x = -1, y = -1; static constexpr float w = 1.f / 36.f; };
template <> struct Vel<8> { static constexpr int x = 1, y = -1; static constexpr float w = 1.f / 36.f; };

// A float-float number hi + lo with |lo| <= ulp(hi)/2.
struct df2 {
    float hi, lo;
};

// Per-lattice constants, precomputed on the host.
struct LatDev {
    int64_t off_f[2];  // element offset of plane 0 of buffers A, B in the population arena
    int64_t off_psi;   // element offset of the psi plane in the psi arena
    int64_t plane;     // population plane stride (elements)
    int32_t nx, ny;
    int32_t pitch;      // population row pitch (elements)
    int32_t gx;         // column of x = 0 inside a population row
    int32_t pitch_psi;  // psi row pitch (floats)
    int32_t gx_psi;     // column of x = 0 inside a psi row
    float omega;        // 1 / tau                                   Eq. (BGKCO)
    float guo;          // 1 - 1/(2 tau)                             Eq. (GFSBGK)
    // F = k_sc psi M1 + k1 (M1.M2) + k2 (M1 tr M2 - M1.M2), i.e. Eq. (IFT) with
    // F^SC of Eq. (SCF), F1 of Eq. (DFTCCC) and F2 of Eq. (DFTCST) expanded:
    float k_sc;         // -2 G / c_s^2                  = -6 G
    float k1;           // (-3/4 eps c_s^2 G)(-2 / c_s^6) = 13.5 eps G
    float k2;           // (sigma - 1) c_s^2 G / c_s^6    = 9 (sigma - 1) G
    float rho0;         // deviation reference (0 for plain FP32 storage)
    int32_t m2_variant; // 0: direct trace; 1: 2 c_s^2 (M0 - psi)
    int32_t lattice;    // index for the status word
    // psi(rho)^2 = (P_EOS - c_s^2 rho)/G = rho (e1 q(rho) - e2 rho - e3),
    // q = (1 + eta + eta^2 - eta^3)/(1 - eta)^3, eta = b rho      Eqs. (DED), (CSEOS)
    double eb, e1, e2, e3;
    df2 fb, f1, f2, f3;  // the same constants as float-float pairs
    float sb, s1, s2, s3; // ... and as floats
    // MRT relaxation rates (Eq. RelaxationMatrix), used by the MRT kernels
    float mrt_s[9];
};

struct StepArgs {
    const LatDev* lats;
    const int4* tiles;  // (lattice, x0, y0, unused)
    int ntiles;
    void* pop;          // population arena
    float* psi;         // psi arena
    uint32_t* status;   // per-lattice fault bits: 1 psi undefined, 2 copy wait timed out,
                        // 4 a staging copy broke the alignment rules (skipped)
    int parity;         // which population buffer holds the current state
    // optional per-lattice step quotas (server chunks): tiles of a lattice with
    // step >= quota[lattice] are skipped; nullptr for handles
    const int* quota;
    int step;
};

// ---- storage traits ---------------------------------------------------------
struct StoreF32 {
    using T = float;
    static constexpr int kGx = 4;  // 16 bytes of ghost columns keep rows aligned
    // read-only load that asks L2 to fetch 256-byte blocks (neighbouring warps
    // read the adjacent segments of the same rows)
    static __device__ __forceinline__ float ld(const float* p) {
        float v;
        asm volatile("ld.global.nc.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(p));
        return v;
    }
    static __device__ __forceinline__ float lds(const float* p) { return *p; }
    static __device__ __forceinline__ float cv(float v) { return v; }
};
struct StoreF16 {
    using T = __half;
    static constexpr int kGx = 8;
    static __device__ __forceinline__ float ld(const __half* p) {
        unsigned short v;
        asm volatile("ld.global.nc.L2::256B.b16 %0, [%1];" : "=h"(v) : "l"(p));
        return __half2float(__ushort_as_half(v));
    }
    static __device__ __forceinline__ float lds(const __half* p) { return __half2float(*p); }
    static __device__ __forceinline__ __half cv(float v) { return __float2half_rn(v); }
};

// Write v at interior site (x, y) and at every periodic image of it that lies
// within GW of the interior (two images per axis when the lattice is
// narrower than 2 GW).  Requires nx, ny >= GW.
template <class T>
__device__ __forceinline__ void store_img(T* plane, int pitch, int gx, int x, int y, int nx,
                                          int ny, T v) {
    T* const row = plane + (int64_t)(y + GY) * pitch + gx;
    row[x] = v;
    const bool xl = x < GW, xh = x >= nx - GW, yl = y < GW, yh = y >= ny - GW;
    if (xl | xh | yl | yh) {
        if (xl) row[x + nx] = v;
        if (xh) row[x - nx] = v;
        if (yl) {
            T* const r = row + (int64_t)ny * pitch;
            r[x] = v;
            if (xl) r[x + nx] = v;
            if (xh) r[x - nx] = v;
        }
        if (yh) {
            T* const r = row - (int64_t)ny * pitch;
            r[x] = v;
            if (xl) r[x + nx] = v;
            if (xh) r[x - nx] = v;
        }
    }
}

// ---- float-float arithmetic (error-free transformations) ---------------------
// TwoSum: Knuth, TAOCP vol. 2; FastTwoSum: Dekker 1971; TwoProd via FMA.
// Intrinsics (__fadd_rn etc.) are never contracted or reordered by nvcc.
__device__ __forceinline__ df2 two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ df2 fast_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df2 df_add(df2 a, df2 b) {
    df2 s = two_sum(a.hi, b.hi);
    df2 t = two_sum(a.lo, b.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = fast_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df2 df_neg(df2 a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df2 df_mul(df2 a, df2 b) {
    float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ df2 df_mul_f(df2 a, float b) {
    float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    e = __fmaf_rn(a.lo, b, e);
    return fast_two_sum(p, e);
}
// Long division with two correction quotients (Bailey's double-double scheme).
__device__ __forceinline__ df2 df_div(df2 a, df2 b) {
    float q1 = __fdiv_rn(a.hi, b.hi);
    df2 r = df_add(a, df_neg(df_mul_f(b, q1)));
    float q2 = __fdiv_rn(r.hi, b.hi);
    r = df_add(r, df_neg(df_mul_f(b, q2)));
    float q3 = __fdiv_rn(r.hi, b.hi);
    df2 q = fast_two_sum(q1, q2);
    return df_add(q, df2{q3, 0.f});
}

// ---- psi(rho), Eqs. (DED) and (CSEOS) --------------------------------------
// psi^2 = (P_EOS - c_s^2 rho)/G = rho (e1 q - e2 rho - e3) with
// q = (1 + eta + eta^2 - eta^3)/(1 - eta)^3, eta = b rho.  Writing
// r = 1/(1 - eta) turns q into the polynomial 1 - 2r + 2r^3 (exact algebra:
// the numerator is 2 - 2s^2 + s^3 in s = 1 - eta), which needs one
// reciprocal instead of a division of two cubics.
// Returns psi and sets ok = false where psi is undefined (rho <= 0 or not
// finite, b rho >= 1, negative radicand).
enum { EOS_F64 = 0, EOS_DF = 1, EOS_F32 = 2 };

template <int P>
__device__ __forceinline__ float eval_psi(const LatDev& L, float rho, bool& ok);

template <>
__device__ __forceinline__ float eval_psi<EOS_F64>(const LatDev& L, float rho, bool& ok) {
    const double r = (double)rho;
    const double s = fma(-L.eb, r, 1.0);
    const double rr = 1.0 / s;
    const double q = fma(2.0 * rr, rr * rr, fma(-2.0, rr, 1.0));
    const double arg = r * fma(L.e1, q, -fma(L.e2, r, L.e3));
    ok = (rho > 0.f) && (s > 0.0) && (arg >= 0.0) && isfinite(arg);
    return sqrtf((float)arg);
}

// 1/s in float-float: one Newton step on the rounded reciprocal.
__device__ __forceinline__ df2 df_rcp(df2 s) {
    const float q = __frcp_rn(s.hi);
    const float e = __fmaf_rn(-s.lo, q, __fmaf_rn(-s.hi, q, 1.f));  // 1 - s q
    return fast_two_sum(q, __fmul_rn(q, e));
}

template <>
__device__ __forceinline__ float eval_psi<EOS_DF>(const LatDev& L, float rho, bool& ok) {
    const df2 br = df_mul_f(L.fb, rho);
    df2 s = two_sum(1.f, -br.hi);  // 1 - b rho
    s = fast_two_sum(s.hi, __fsub_rn(s.lo, br.lo));
    const df2 r = df_rcp(s);
    const df2 r3 = df_mul(df_mul(r, r), r);
    // q = 1 - 2 r + 2 r^3 (doubling is exact)
    const df2 q = df_add(df_add(df2{1.f, 0.f}, df2{-2.f * r.hi, -2.f * r.lo}),
                         df2{2.f * r3.hi, 2.f * r3.lo});
    const df2 t = df_add(df_mul_f(L.f2, rho), L.f3);
    const df2 inner = df_add(df_mul(L.f1, q), df_neg(t));
    const df2 arg = df_mul_f(inner, rho);
    ok = (rho > 0.f) && (s.hi > 0.f) && (arg.hi >= 0.f) && isfinite(arg.hi);
    return sqrtf(arg.hi);
}

template <>
__device__ __forceinline__ float eval_psi<EOS_F32>(const LatDev& L, float rho, bool& ok) {
    const float s = fmaf(-L.sb, rho, 1.f);
    const float rr = 1.f / s;
    const float q = fmaf(2.f * rr, rr * rr, fmaf(-2.f, rr, 1.f));
    const float arg = rho * fmaf(L.s1, q, -fmaf(L.s2, rho, L.s3));
    ok = (rho > 0.f) && (s > 0.f) && (arg >= 0.f) && isfinite(arg);
    return sqrtf(arg);
}

// ---- force of Eq. (IFT) from the nine psi values around a site ------------
// p[0] = psi(x); p[i] = psi(x + c_i).
// M1 and M2 (Eqs. FOMED, SOMED) with the D2Q9 weights multiplied out.
struct Force {
    float x, y;
};
__device__ __forceinline__ Force site_force(const LatDev& L, float p0, float pE, float pN,
                                            float pW, float pS, float pNE, float pNW,
                                            float pSW, float pSE) {
    const float m1x = (4.f * (pE - pW) + (pNE - pNW) + (pSE - pSW)) * (1.f / 36.f);
    const float m1y = (4.f * (pN - pS) + (pNE + pNW) - (pSW + pSE)) * (1.f / 36.f);
    const float sd = (pNE + pNW) + (pSW + pSE);
    const float sx = pE + pW, sy = pN + pS;
    const float m2xx = (-8.f * p0 + 4.f * sx - 2.f * sy + sd) * (1.f / 54.f);
    const float m2yy = (-8.f * p0 + 4.f * sy - 2.f * sx + sd) * (1.f / 54.f);
    const float m2xy = ((pNE - pNW) + (pSW - pSE)) * (1.f / 36.f);
    const float tr = L.m2_variant ? (-20.f * p0 + 4.f * (sx + sy) + sd) * (1.f / 54.f)
                                  : (m2xx + m2yy);
    const float ax = m1x * m2xx + m1y * m2xy;  // M1_b M2_ab
    const float ay = m1x * m2xy + m1y * m2yy;
    Force F;
    F.x = L.k_sc * p0 * m1x + L.k1 * ax + L.k2 * (m1x * tr - ax);
    F.y = L.k_sc * p0 * m1y + L.k1 * ay + L.k2 * (m1y * tr - ay);
    return F;
}

// ---- BGK collision with Guo forcing for direction I ------------------------
// g: stored (deviation) population; returns the post-collision value.
// f^eq - w rho0 = w (drho + rho (3 cu + 9/2 cu^2 - 3/2 u^2))          Eq. (SEDF)
// S = (1 - 1/2tau) w (3 cF + 9 cF cu - 3 F.u)                          Eqs. (GFS), (GFSBGK)
template <int I>
__device__ __forceinline__ float bgk_guo(float g, float drho, float rho, float ux, float uy,
                                         float usq, float Fx, float Fy, float Fu, float omega,
                                         float guo) {
    constexpr float w = Vel<I>::w;
    const float cu = (float)Vel<I>::x * ux + (float)Vel<I>::y * uy;
    const float cF = (float)Vel<I>::x * Fx + (float)Vel<I>::y * Fy;
    const float feq = w * (drho + rho * (3.f * cu + 4.5f * cu * cu - 1.5f * usq));
    const float src = guo * w * (3.f * cF + 9.f * cF * cu - 3.f * Fu);
    return g + omega * (feq - g) + src;
}

// Per-lattice constants of one site update, held in registers for a tile.
struct SiteConsts {
    float omega, guo, rho0, k_sc, k1, k2;
    int m2v;
};
__device__ __forceinline__ SiteConsts site_consts(const LatDev& L) {
    return SiteConsts{L.omega, L.guo, L.rho0, L.k_sc, L.k1, L.k2, L.m2_variant};
}

// One site of the collision pass: pulled (deviation) populations g[0..8]
// and psi at x + c_i (p[0] = psi(x), then E, N, W, S, NE, NW, SW, SE) in,
// post-collision deviations o[0..8] out.
//   rho, j     Eqs. (FD), (FMD)
//   F          Eq. (IFT) via site_force
//   f*_i       Eqs. (BGKCO), (SEDF), (GFS), (GFSBGK), with opposite
//              directions sharing their terms: for c and -c,
//              f^eq = w (base + rho cu (3 +- 9/2 cu)) with base = drho - 3/2 rho u^2,
//              S    = gu w (9 cF cu +- 3 cF - 3 F.u);
// the rest population f*_0 takes what mass conservation leaves (in exact
// arithmetic the same number; it keeps the FP32 weights, whose sum is not
// exactly 1, from adding a biased mass error every step).
__device__ __forceinline__ void collide_site(const SiteConsts& C, const float g[9],
                                             const float p[9], float o[9]) {
    const float drho = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
    const float rho = drho + C.rho0;
    const float jx = (g[1] - g[3]) + (g[5] - g[6]) + (g[8] - g[7]);
    const float jy = (g[2] - g[4]) + (g[5] + g[6]) - (g[7] + g[8]);
    LatDev dummy;  // site_force reads only the force coefficients and the trace flag
    dummy.k_sc = C.k_sc;
    dummy.k1 = C.k1;
    dummy.k2 = C.k2;
    dummy.m2_variant = C.m2v;
    const Force F = site_force(dummy, p[0], p[1], p[2], p[3], p[4], p[5], p[6], p[7], p[8]);
    const float inv = __frcp_rn(rho);
    const float ux = fmaf(0.5f, F.x, jx) * inv;  // Eq. (FMD)
    const float uy = fmaf(0.5f, F.y, jy) * inv;
    const float usq = ux * ux + uy * uy;
    const float f3u = 3.f * (F.x * ux + F.y * uy);
    const float base = drho - 1.5f * rho * usq;
    const float om = C.omega;
    const float ga = C.guo * (1.f / 9.f), gd = C.guo * (1.f / 36.f);
    float s1 = 0.f;
    // one pair of opposite directions (I, J = opposite of I), weight w, guo weight gw
#define PPLBM_PAIR(I, J, W, GW, CU, CF)                                             \
    {                                                                               \
        const float cu = (CU), cF = (CF);                                           \
        const float t = rho * cu;                                                   \
        const float a = 4.5f * t * cu, b = 3.f * t;                                 \
        const float s2 = 9.f * cF * cu - f3u, s3 = 3.f * cF;                        \
        const float fi = (W) * (base + a + b), fj = (W) * (base + a - b);          \
        const float oi = fmaf(om, fi - g[I], g[I]) + (GW) * (s2 + s3);              \
        const float oj = fmaf(om, fj - g[J], g[J]) + (GW) * (s2 - s3);              \
        o[I] = oi;                                                                  \
        o[J] = oj;                                                                  \
        s1 += oi + oj;                                                              \
    }
    PPLBM_PAIR(1, 3, 1.f / 9.f, ga, ux, F.x)
    PPLBM_PAIR(2, 4, 1.f / 9.f, ga, uy, F.y)
    PPLBM_PAIR(5, 7, 1.f / 36.f, gd, ux + uy, F.x + F.y)
    PPLBM_PAIR(6, 8, 1.f / 36.f, gd, uy - ux, F.y - F.x)
#undef PPLBM_PAIR
    o[0] = drho - s1;
}

// MRT collision (Eq. MRTCO) with Guo forcing in moment space (Eq. GFSMRT),
// for the Gram-Schmidt matrix M of Appendix A.  Same inputs and outputs as
// collide_site.  Moments of the stored deviations: m(f) = M g + rho0 M w with
// M w = (1, -2, 1, 0, ..., 0).  Post-collision moments
//   m* = m - Lambda (m - m^eq) + (I - Lambda/2) M S
// with m^eq and M S the vectors printed in Appendix A (rho u is the
// force-shifted momentum of Eq. FMD).  Back to populations with
// M^-1 = M^T D^-1, D = diag(9, 36, 36, 6, 12, 6, 12, 4, 4) (the rows of M
// are orthogonal); the rest population again from mass conservation.
__device__ __forceinline__ void collide_site_mrt(const SiteConsts& C, const float* s,
                                                 const float g[9], const float p[9],
                                                 float o[9]) {
    const float drho = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
    const float rho = drho + C.rho0;
    const float jx = (g[1] - g[3]) + (g[5] - g[6]) + (g[8] - g[7]);
    const float jy = (g[2] - g[4]) + (g[5] + g[6]) - (g[7] + g[8]);
    LatDev dummy;
    dummy.k_sc = C.k_sc;
    dummy.k1 = C.k1;
    dummy.k2 = C.k2;
    dummy.m2_variant = C.m2v;
    const Force F = site_force(dummy, p[0], p[1], p[2], p[3], p[4], p[5], p[6], p[7], p[8]);
    const float inv = __frcp_rn(rho);
    const float rux = fmaf(0.5f, F.x, jx), ruy = fmaf(0.5f, F.y, jy);  // rho u, Eq. (FMD)
    const float ux = rux * inv, uy = ruy * inv;
    const float usq = ux * ux + uy * uy;
    const float uF = ux * F.x + uy * F.y;
    // moments of f (deviations shifted by rho0 M w)
    const float sa = (g[1] + g[2]) + (g[3] + g[4]), sd = (g[5] + g[6]) + (g[7] + g[8]);
    const float m1 = (-4.f * g[0] - sa + 2.f * sd) - 2.f * C.rho0;
    const float m2 = (4.f * g[0] - 2.f * sa + sd) + C.rho0;
    const float m4 = (-2.f * g[1] + 2.f * g[3]) + ((g[5] - g[6]) + (g[8] - g[7]));
    const float m6 = (-2.f * g[2] + 2.f * g[4]) + ((g[5] + g[6]) - (g[7] + g[8]));
    const float m7 = (g[1] - g[2]) + (g[3] - g[4]);
    const float m8 = (g[5] - g[6]) + (g[7] - g[8]);
    // m* = m - s (m - meq) + (1 - s/2) Sbar, component by component
    const float r3u2 = 3.f * rho * usq;
    const float p1 = m1 - s[1] * (m1 - (-2.f * rho + r3u2)) + (1.f - 0.5f * s[1]) * (6.f * uF);
    const float p2 = m2 - s[2] * (m2 - (rho - r3u2)) + (1.f - 0.5f * s[2]) * (-6.f * uF);
    const float p3 = jx - s[3] * (jx - rux) + (1.f - 0.5f * s[3]) * F.x;
    const float p4 = m4 - s[4] * (m4 + rux) + (1.f - 0.5f * s[4]) * (-F.x);
    const float p5 = jy - s[5] * (jy - ruy) + (1.f - 0.5f * s[5]) * F.y;
    const float p6 = m6 - s[6] * (m6 + ruy) + (1.f - 0.5f * s[6]) * (-F.y);
    const float p7 = m7 - s[7] * (m7 - rho * (ux * ux - uy * uy)) +
                     (1.f - 0.5f * s[7]) * (2.f * (ux * F.x - uy * F.y));
    const float p8 = m8 - s[8] * (m8 - rho * ux * uy) + (1.f - 0.5f * s[8]) * (ux * F.y + uy * F.x);
    // back to deviations: subtract rho0 M w from the moments, then M^T D^-1
    const float q0 = drho * (1.f / 9.f);
    const float q1 = (p1 + 2.f * C.rho0) * (1.f / 36.f);
    const float q2 = (p2 - C.rho0) * (1.f / 36.f);
    const float q3 = p3 * (1.f / 6.f), q4 = p4 * (1.f / 12.f);
    const float q5 = p5 * (1.f / 6.f), q6 = p6 * (1.f / 12.f);
    const float q7 = p7 * 0.25f, q8 = p8 * 0.25f;
    const float ax = q0 - q1 - 2.f * q2;  // common part of the axis directions
    const float dg = q0 + 2.f * q1 + q2;  // common part of the diagonals
    o[1] = ax + q3 - 2.f * q4 + q7;
    o[2] = ax + q5 - 2.f * q6 - q7;
    o[3] = ax - q3 + 2.f * q4 + q7;
    o[4] = ax - q5 + 2.f * q6 - q7;
    o[5] = dg + q3 + q4 + q5 + q6 + q8;
    o[6] = dg - q3 - q4 + q5 + q6 - q8;
    o[7] = dg - q3 - q4 - q5 - q6 + q8;
    o[8] = dg + q3 + q4 - q5 - q6 - q8;
    o[0] = drho - (((o[1] + o[2]) + (o[3] + o[4])) + ((o[5] + o[6]) + (o[7] + o[8])));
}

// Store the nine outputs of site (x, y): interior sites with plain stores,
// sites within GW of an edge also into their periodic images.
template <class S>
__device__ __forceinline__ void store_site(typename S::T* o, int64_t plane, int pitch, int gx,
                                           int x, int y, int nx, int ny, const float v[9]) {
    const bool interior = (x >= GW) & (x < nx - GW) & (y >= GW) & (y < ny - GW);
    if (interior) {
        typename S::T* q = o + (int64_t)(y + GY) * pitch + (x + gx);
#pragma unroll
        for (int i = 0; i < 9; ++i) q[i * plane] = S::cv(v[i]);
    } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) store_img(o + i * plane, pitch, gx, x, y, nx, ny, S::cv(v[i]));
    }
}

}  // namespace pplbm
