// lbm_device.cuh -- device-side data layout and per-site arithmetic of the
// D2Q9 pseudopotential step (arXiv 2003.07968) for sm_103a.
//
// Layout in HBM (per lattice, per population buffer):
//   nine SoA planes, one per velocity c_i (Eq. VelocitySet order), each a
//   pitched 2-D array with a ghost frame: rows [-GY, ny+GY), columns
//   [-gx, pitch-gx).  Ghost sites within GW of the interior hold periodic
//   images, written by the same kernel that writes the interior site, so
//   readers never wrap indices (the batch form writes only the planes a
//   step reads at each image: store_images).  Two population buffers (A/B)
//   alternate between steps; a float psi plane with the same ghost frame
//   sits beside.
//   The buffers hold POST-collision, PRE-streaming populations f*; a step
//   pulls f_i(x) = f*_i(x - c_i) (streaming of Eq. TLBE in pull form).
//
// What a buffer stores (rest-referenced deviations): for every site y,
//   plane 0:  R(y)   = f*_0(y) - w_0 rho0,
//   plane i:  G_i(y) = (f*_i(y) - w_i rho0) - c'_i R(y) + E(y)/8,  i = 1..8,
// with c'_i = w_i / w_0 (1/4 on the axes, 1/16 on the diagonals: exact in
// any binary format) and rho0 the lattice's deviation reference.  Near
// equilibrium f*_i ~ c'_i f*_0, so the eight G_i are small numbers and keep
// their own rounding small; the one large stored number, R, is rounded once,
// and E = 9/4 (exact R - stored R) puts that rounding back into the G_i, so
// the stored mass of a site, rho0 + 9/4 R + sum_i G_i, is the mass the
// collision conserved up to roundings of small numbers.  Storing each f*_i
// (or f*_i - w_i rho0) on its own rounds nine large numbers per site, and in
// a uniform phase every site rounds them alike: a bias that is the same
// across a whole phase and acts like a pressure offset between liquid and
// vapour, moving interfaces (measured: 2.6e-5 relative density error after
// 1000 steps on a 512^2 droplet, against 3.5e-6 with this form, both against
// the FP64 step).
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace pplbm {

constexpr int GW = 2;  // depth of the periodic images kept around the interior
constexpr int GY = 2;  // ghost rows above and below

// D2Q9 velocity set, Eq. (VelocitySet); weights from the text after Eq. (SEDF).
__device__ __constant__ static const int kCx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__device__ __constant__ static const int kCy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
// the same directions as compile-time functions of the plane index
__host__ __device__ constexpr int plane_cy(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__host__ __device__ constexpr int plane_cx(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}

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

// c'_i = w_i / w_0, the ratio between a moving population's equilibrium and
// the rest population's (exact: 1/4 and 1/16).
__host__ __device__ constexpr float cref(int i) { return i == 0 ? 1.f : (i <= 4 ? 0.25f : 0.0625f); }

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
    float omega;        // 1 / tau, rounded to FP32                  Eq. (BGKCO)
    float guo;          // 1 - omega/2 (exact from the FP32 omega)   Eq. (GFSBGK)
    // F = k_sc psi M1 + k1 (M1.M2) + k2 (M1 tr M2 - M1.M2), i.e. Eq. (IFT) with
    // F^SC of Eq. (SCF), F1 of Eq. (DFTCCC) and F2 of Eq. (DFTCST) expanded:
    float k_sc;         // -2 G / c_s^2                  = -6 G
    float k1;           // (-3/4 eps c_s^2 G)(-2 / c_s^6) = 13.5 eps G
    float k2;           // (sigma - 1) c_s^2 G / c_s^6    = 9 (sigma - 1) G
    // ... with the scale factors of the integer stencils folded in (site_force)
    float fsc, fk2, fkd;  // k_sc / 36, k2 / 1944, (k1 - k2) / 1944
    // BGK + Guo per weight class, axis w = 1/9 (a) and diagonal w = 1/36 (d),
    // as collide_bgk uses them; all but rw0, rg0 are exact functions of the
    // FP32 omega (1 - omega, omega/2, ... are exact in FP32)
    float om1;          // 1 - omega
    float rw0, rg0;     // omega w_0, -3 guo w_0 (the rest population's update)
    float ra, rd;       // 9/2 omega w = omega/2, omega/8
    float ga9, gd9;     // 9 guo w = guo, guo/4
    float rho0;         // deviation reference (0 for plain FP32 storage)
    int32_t m2_variant; // 0: direct trace; 1: 2 c_s^2 (M0 - psi)
    int32_t eos_kind;   // 0: Carnahan-Starling, Eq. (CSEOS); 1: van der Waals
    int32_t lattice;    // index for the status word
    int32_t row0;       // row of the arena's row space where this lattice's ghost
                        // row -GY starts (off_f[0] = row0 * pitch), or -1
    // psi(rho)^2 = (P_EOS - c_s^2 rho)/G = rho (e1 q(rho) - e2 rho - e3),
    // eta = b rho, q = (1 + eta + eta^2 - eta^3)/(1 - eta)^3 (Carnahan-Starling,
    // Eq. CSEOS) or q = 1/(1 - eta) (van der Waals)               Eq. (DED)
    double eb, e1, e2, e3;
    df2 fb, f2, fc0, fC1;  // b, e2, c0 = e1 - e3, C1 (2 b e1; van der Waals b e1)
                           // as float-float pairs
    float sb, s1, s2, s3;  // b, e1, e2, e3 as floats
    float zero;            // 0, as a value the compiler cannot see (Eos<EOS_DF>)
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
    // failure-detection test: tile + 1 whose staging copy the single pass
    // skips, so that the consumers' bounded wait for it runs out (0: none)
    int starve = 0;
    // clock budget of the single pass's waits (SM cycles): kWaitBudgetCycles,
    // or kTestWaitBudgetCycles in the launch that carries an armed test.  A
    // kernel parameter, read only once a wait has not finished at once
    long long wait_cycles = 4000000000LL;
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
    // the value a float becomes once stored and loaded again
    static __device__ __forceinline__ float rt(float v) { return v; }
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
    static __device__ __forceinline__ float rt(float v) { return __half2float(__float2half_rn(v)); }
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

// ---- lane-parallel FP32 -------------------------------------------------------
// The site arithmetic below is written once over V = float (one site) or
// V = float2 (two sites).  For float2 every operation is one of the paired
// FP32 instructions of sm_100 and later (add/sub/mul/fma .f32x2: two lanes per
// issue slot); for float it is the scalar instruction.  Both are written as
// PTX with an explicit .rn rounding modifier, which the compiler's optimiser
// cannot see through.  Two facts measured on sm_103a shape the code:
//  - the code generator keeps scalar .rn operations as written, but fuses a
//    paired multiply into a following paired add or subtract even with .rn;
//    so no product of a paired multiply ever feeds a paired add here:
//    products enter FMAs as multiplicands or addends, and a product that
//    must be added is formed as an FMA with a zero addend the compiler
//    cannot see (the float-float EOS);
//  - the CUDA rounding intrinsics (__fadd_rn ...) are not enough either:
//    a TwoSum error term built from them folded to zero.
// Every operation is then one IEEE round-to-nearest step per lane, in the
// order written, and a site gets bitwise the same result whichever lane
// count, tile or kernel computes it.
__device__ __forceinline__ float vadd(float a, float b) {
    float d;
    asm("add.rn.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}
__device__ __forceinline__ float vsub(float a, float b) {
    float d;
    asm("sub.rn.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}
__device__ __forceinline__ float vmul(float a, float b) {
    float d;
    asm("mul.rn.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}
__device__ __forceinline__ float vfma(float a, float b, float c) {
    float d;
    asm("fma.rn.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
#define PPLBM_F32X2_BINARY(NAME, OP)                                                       \
    __device__ __forceinline__ float2 NAME(float2 a, float2 b) {                          \
        float2 d;                                                                          \
        asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t" \
            OP " rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"                                  \
            : "=f"(d.x), "=f"(d.y)                                                         \
            : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));                                     \
        return d;                                                                          \
    }
PPLBM_F32X2_BINARY(vadd, "add.rn.f32x2")
PPLBM_F32X2_BINARY(vsub, "sub.rn.f32x2")
PPLBM_F32X2_BINARY(vmul, "mul.rn.f32x2")
#undef PPLBM_F32X2_BINARY
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mov.b64 rc, {%6, %7};\n\tfma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}

template <class V> struct Lanes;
template <> struct Lanes<float> {
    static constexpr int n = 1;
    static __device__ __forceinline__ float set(float c) { return c; }
    static __device__ __forceinline__ float get(float v, int) { return v; }
    static __device__ __forceinline__ void put(float& v, int, float c) { v = c; }
};
template <> struct Lanes<float2> {
    static constexpr int n = 2;
    static __device__ __forceinline__ float2 set(float c) { return make_float2(c, c); }
    static __device__ __forceinline__ float get(float2 v, int k) { return k ? v.y : v.x; }
    static __device__ __forceinline__ void put(float2& v, int k, float c) {
        if (k)
            v.y = c;
        else
            v.x = c;
    }
};
// vector type of a thread that handles SPT sites: pairs when SPT is even
template <int SPT> struct LaneOf { using V = typename std::conditional<SPT % 2 == 0, float2, float>::type; };

// ---- the pulled state of a site ------------------------------------------------
// Site x pulls f_i(x) = f*_i(x - c_i); as deviations from w_i rho0 these are
// g_0 = R(x) and g_i = G_i(x - c_i) + c'_i R(x - c_i).  The step works with
//   r0  = R(x),
//   h_i = g_i - c'_i r0 = G_i(x - c_i) + c'_i (R(x - c_i) - R(x)),   i = 1..8,
//   D   = sum_i h_i,
// so that the density deviation is drho = sum_i g_i = 9/4 r0 + D (c'_0 + sum_i
// c'_i = 9/4) and the momentum is sum_i c_i g_i = sum_i c_i h_i (the c'_i r0
// cancel in opposite pairs).  Near equilibrium the h_i and D are small, and
// so is every number the collision then forms.
template <class V>
struct Site {
    V r0, D;
    V h[9];  // h[1..8]
};

// The site from R[i] = R(x - c_i) (R[0] = R(x)) and Gs[i] = G_i(x - c_i),
// in the one order of operations that every kernel uses.
template <class V>
__device__ __forceinline__ Site<V> make_site(const V R[9], const V Gs[9]) {
    using Ln = Lanes<V>;
    Site<V> s;
    s.r0 = R[0];
#pragma unroll
    for (int i = 1; i < 9; ++i) s.h[i] = vfma(Ln::set(cref(i)), vsub(R[i], R[0]), Gs[i]);
    s.D = vadd(vadd(vadd(s.h[1], s.h[2]), vadd(s.h[3], s.h[4])),
               vadd(vadd(s.h[5], s.h[6]), vadd(s.h[7], s.h[8])));
    return s;
}

// rho = rho0 + 9/4 r0 + D (Eq. FD).
template <class V>
__device__ __forceinline__ V site_rho(const Site<V>& s, float rho0) {
    using Ln = Lanes<V>;
    return vadd(vfma(Ln::set(2.25f), s.r0, s.D), Ln::set(rho0));
}

// The hardware approximations (one MUFU instruction each, flush to zero):
// fixed functions of their input, so every kernel gets the same bits.
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// 1/x for normal x > 0 (the EOS and the collision): the hardware
// approximation r per lane, then one Newton-Raphson step for f(r) = 1/r - x,
//   r' = r + r (1 - x r),
// two FMAs on the paired pipe (Muller et al., Handbook of Floating-Point
// Arithmetic, Newton-Raphson based division).  The step squares the
// approximation's relative error, so r' is within about 1 ulp of 1/x
// (tested against correctly rounded reciprocals, lbm_selfcheck_arith).
template <class V>
__device__ __forceinline__ V vrcp(V x) {
    using Ln = Lanes<V>;
    V r;
#pragma unroll
    for (int k = 0; k < Ln::n; ++k) Ln::put(r, k, rcp_approx(Ln::get(x, k)));
    const V e = vfma(vmul(x, Ln::set(-1.f)), r, Ln::set(1.f));  // 1 - x r
    return vfma(r, e, r);
}

// sqrt(a) for finite a >= 0 (psi): the hardware reciprocal square root y
// per lane, s = a y, then one Newton step on the square root (Markstein's
// method),
//   s' = s + (y / 2)(a - s^2),
// on the paired pipe.  a below 2^-100 is scaled by 2^100 first and the root
// by 2^-50 after (both exact), and a = 0 gives 0, so the flush to zero of the
// approximation never shows.  Within about 1 ulp of sqrt(a) (tested against
// correctly rounded roots, lbm_selfcheck_arith).
template <class V>
__device__ __forceinline__ V vsqrt(V a) {
    using Ln = Lanes<V>;
    V as, y, sc;
#pragma unroll
    for (int k = 0; k < Ln::n; ++k) {
        const float x = Ln::get(a, k);
        const bool tiny = x < 0x1p-100f;
        const float xs = tiny ? x * 0x1p100f : x;
        Ln::put(as, k, xs);
        Ln::put(sc, k, tiny ? 0x1p-50f : 1.f);
        Ln::put(y, k, rsqrt_approx(xs));
    }
    const V s = vmul(as, y);
    const V e = vfma(vmul(s, Ln::set(-1.f)), s, as);  // a - s^2
    const V r = vmul(vfma(vmul(y, Ln::set(0.5f)), e, s), sc);
    V out;
#pragma unroll
    for (int k = 0; k < Ln::n; ++k) Ln::put(out, k, Ln::get(a, k) == 0.f ? 0.f : Ln::get(r, k));
    return out;
}

// ---- psi(rho), Eqs. (DED) and (CSEOS) --------------------------------------
// psi^2 = (P_EOS - c_s^2 rho)/G = rho (e1 q - e2 rho - e3) with
// q = (1 + eta + eta^2 - eta^3)/(1 - eta)^3, eta = b rho.  With r = 1/(1 - eta)
// one has eta r = r - 1 and (2 - eta) r = 1 + r, so q = 1 - 2r + 2r^3 =
// 1 + 2 eta r^2 (1 + r) exactly, and
//   psi^2 / rho = c0 + rho (C1 r^2 (1 + r) - e2),   c0 = e1 - e3,  C1 = 2 b e1.
// The van der Waals equation behind the same psi (eos_kind 1) has q = r =
// 1 + eta r, so psi^2 / rho = c0 + rho (C1 r - e2) with C1 = b e1: the same
// sums with r in place of r^2 (1 + r).
// For the Carnahan-Starling constants at 0.55 <= T_r <= 1 and rho <= 3.6 no sum
// here cancels by more than a factor of about 8, and the float-float version
// (below) keeps about 43 significant bits of the radicand.
// A lane is valid when rho > 0, b rho < 1 and the radicand is finite and
// positive and normal (at least 2^-126); an invalid lane gets psi = NaN and, if its
// bit in `live` is set, raises status bit 1 of its lattice (lanes without a
// site are not live).
enum { EOS_F64 = 0, EOS_DF = 1, EOS_F32 = 2 };

// sqrt of the EOS radicand: vsqrt without its scaling of tiny arguments
// (the same operations, so the same bits, for a >= 2^-100; down to 2^-126
// the residual a - s^2 is exact in the fused multiply-add, so the root stays
// within about 1 ulp).  A subnormal radicand (the approximation flushes it
// to zero), zero or a negative one gives a root that is not finite, which
// psi_finish reports as psi undefined.
template <class V>
__device__ __forceinline__ V vsqrt_eos(V a) {
    using Ln = Lanes<V>;
    V y;
#pragma unroll
    for (int k = 0; k < Ln::n; ++k) Ln::put(y, k, rsqrt_approx(Ln::get(a, k)));
    const V s = vmul(a, y);
    const V e = vfma(vmul(s, Ln::set(-1.f)), s, a);  // a - s^2
    return vfma(vmul(y, Ln::set(0.5f)), e, s);
}

template <class V>
__device__ __forceinline__ V psi_finish(const LatDev& L, V rho, V s, V arg, uint32_t* status,
                                        unsigned live) {
    const V root = vsqrt_eos(arg);
    V psi;
    unsigned bad = 0;
#pragma unroll
    for (int k = 0; k < Lanes<V>::n; ++k) {
        const float q = Lanes<V>::get(root, k);
        const bool ok =
            (Lanes<V>::get(rho, k) > 0.f) && (Lanes<V>::get(s, k) > 0.f) && (fabsf(q) < INFINITY);
        bad |= (unsigned)!ok << k;
        Lanes<V>::put(psi, k, ok ? q : __int_as_float(0x7fc00000));
    }
    if (bad & live) atomicOr(status + L.lattice, 1u);
    return psi;
}

template <int P>
struct Eos;

// Native FP64, lane by lane (the FP64 pipe has no paired form).
template <>
struct Eos<EOS_F64> {
    template <class V>
    static __device__ __forceinline__ V psi(const LatDev& L, V rho, uint32_t* status,
                                            unsigned live = ~0u) {
        V s, arg;
#pragma unroll
        for (int k = 0; k < Lanes<V>::n; ++k) {
            const double r = (double)Lanes<V>::get(rho, k);
            const double sd = fma(-L.eb, r, 1.0);
            const double rr = 1.0 / sd;
            const double q = L.eos_kind ? rr : fma(2.0 * rr, rr * rr, fma(-2.0, rr, 1.0));
            const double a = r * fma(L.e1, q, -fma(L.e2, r, L.e3));
            Lanes<V>::put(s, k, sd > 0.0 ? 1.f : -1.f);
            Lanes<V>::put(arg, k, (float)a);
        }
        return psi_finish(L, rho, s, arg, status, live);
    }
};

// Float-float: TwoProd by FMA, TwoSum where signs may differ, FastTwoSum where
// the larger operand is known, one Newton step on the rounded reciprocal.
// Runtime negations are explicit products by -1 (there is no paired negate).
// Every product that feeds an add (p, rl, Bh, wh) is formed as an FMA with a
// zero addend the compiler cannot see (LatDev::zero): the code generator
// fuses a paired multiply into a following paired add even with .rn
// (measured on sm_103a), which would break the error-free transformations,
// but it cannot fuse an FMA.
template <>
struct Eos<EOS_DF> {
    // psi^2 = rho (hh + hl) before its one rounding to FP32, and
    // sh = 1 - b rho (rounded), for psi() and for the self-check of the radicand
    template <class V>
    static __device__ __forceinline__ void radicand(const LatDev& L, V rho, V& sh, V& hh, V& hl) {
        using Ln = Lanes<V>;
        const V one = Ln::set(1.f), mone = Ln::set(-1.f), z0 = Ln::set(L.zero);
        // b rho = p - en
        const V p = vfma(Ln::set(L.fb.hi), rho, z0);
        V en = vfma(Ln::set(-L.fb.hi), rho, p);
        en = vfma(Ln::set(-L.fb.lo), rho, en);
        // s = 1 - b rho = sh + sl  (FastTwoSum, 1 > b rho)
        sh = vsub(one, p);
        const V sl = vadd(vsub(vsub(one, sh), p), en);
        // r = 1/s = q - rl  (q the rounded 1/sh, one Newton step)
        const V q = vrcp(sh);
        V t = vfma(sh, q, mone);
        t = vfma(sl, q, t);
        const V rl = vfma(q, t, z0);
        // 1 + r = oh + ol  (FastTwoSum, q >= 1)
        const V oh = vadd(q, one);
        const V ol = vsub(vadd(vsub(q, oh), one), rl);
        V Ah, Ae;
        if (L.eos_kind) {
            // van der Waals: A = r = q - rl
            Ah = q;
            Ae = vmul(rl, mone);
        } else {
            // r^2 = r2h + r2l
            const V nq = vmul(q, mone);
            const V r2h = vmul(q, q), nr2h = vmul(nq, q);
            const V r2l = vfma(vmul(q, Ln::set(-2.f)), rl, vfma(q, q, nr2h));
            // A = r^2 (1 + r) = Ah + Ae
            Ah = vmul(r2h, oh);
            Ae = vfma(r2h, oh, vmul(nr2h, oh));
            Ae = vfma(r2h, ol, Ae);
            Ae = vfma(r2l, oh, Ae);
        }
        // C1 A = Bh - nBl
        const V Bh = vfma(Ln::set(L.fC1.hi), Ah, z0);
        V nBl = vfma(Ln::set(-L.fC1.hi), Ah, Bh);
        nBl = vfma(Ln::set(-L.fC1.hi), Ae, nBl);
        nBl = vfma(Ln::set(-L.fC1.lo), Ah, nBl);
        // v = C1 A - e2 = vh + vl  (TwoSum on the leading parts: they may cancel)
        const V ne2h = Ln::set(-L.f2.hi);
        const V vh = vadd(Bh, ne2h);
        const V bb = vsub(vh, Bh);
        const V ve = vadd(vsub(Bh, vsub(vh, bb)), vsub(ne2h, bb));
        const V vl = vadd(vsub(ve, nBl), Ln::set(-L.f2.lo));
        // w = rho v = wh + we
        const V wh = vfma(vh, rho, z0);
        V we = vfma(vh, rho, vmul(vh, vmul(rho, mone)));
        we = vfma(vl, rho, we);
        // c0 + w = hh + hl: FastTwoSum for Carnahan-Starling, whose c0 has at
        // least the exponent of w wherever psi is defined; TwoSum for van der
        // Waals, whose w outgrows c0 as b rho -> 1
        const V c0h = Ln::set(L.fc0.hi);
        hh = vadd(c0h, wh);
        V e;
        if (L.eos_kind) {
            const V bw = vsub(hh, c0h);
            e = vadd(vsub(c0h, vsub(hh, bw)), vsub(wh, bw));
        } else {
            e = vadd(vsub(c0h, hh), wh);
        }
        hl = vadd(e, vadd(Ln::set(L.fc0.lo), we));
    }
    template <class V>
    static __device__ __forceinline__ V psi(const LatDev& L, V rho, uint32_t* status,
                                            unsigned live = ~0u) {
        V sh, hh, hl;
        radicand(L, rho, sh, hh, hl);
        return psi_finish(L, rho, sh, vfma(rho, hh, vmul(rho, hl)), status, live);
    }
};

// Plain FP32 (selectable; no extended precision).
template <>
struct Eos<EOS_F32> {
    template <class V>
    static __device__ __forceinline__ V psi(const LatDev& L, V rho, uint32_t* status,
                                            unsigned live = ~0u) {
        using Ln = Lanes<V>;
        const V one = Ln::set(1.f);
        const V s = vfma(Ln::set(-L.sb), rho, one);
        const V rr = vrcp(s);
        const V q = L.eos_kind ? rr : vfma(vadd(rr, rr), vmul(rr, rr), vfma(Ln::set(-2.f), rr, one));
        const V inner = vfma(Ln::set(L.s1), q, vfma(Ln::set(-L.s2), rho, Ln::set(-L.s3)));
        return psi_finish(L, rho, s, vmul(rho, inner), status, live);
    }
};

// ---- force of Eq. (IFT) from the nine psi values around a site ------------
// p[0] = psi(x); p[i] = psi(x + c_i), i = E, N, W, S, NE, NW, SW, SE.
// With M1 and M2 of Eqs. (FOMED), (SOMED) written as integer stencils
// m1' = 36 M1, m2'_xx = 54 M2_xx, m2'_yy = 54 M2_yy, m2''_xy = 54 M2_xy,
// tr' = 54 tr M2 (either trace variant), the force
//   F = k_sc psi M1 + k1 M1.M2 + k2 (M1 tr M2 - M1.M2)
// becomes F = m1' (fsc psi + fk2 tr') + fkd (m1'.m2'), with fsc = k_sc/36,
// fk2 = k2/1944, fkd = (k1 - k2)/1944 (LatDev).
struct SiteConsts {
    float rho0, om1, rw0, rg0, ra, rd, ga9, gd9, omega, guo, fsc, fk2, fkd;
    int m2v;
    float zero;  // 0, as a value the compiler cannot see (LatDev::zero)
};

template <class V>
__device__ __forceinline__ void site_force(const SiteConsts& C, const V p[9], V& Fx, V& Fy) {
    using Ln = Lanes<V>;
    const V four = Ln::set(4.f);
    const V dEW = vsub(p[1], p[3]), dNS = vsub(p[2], p[4]);
    const V a = vsub(p[5], p[7]), b = vsub(p[6], p[8]);
    const V m1x = vfma(four, dEW, vsub(a, b));
    const V m1y = vfma(four, dNS, vadd(a, b));
    const V sx = vadd(p[1], p[3]), sy = vadd(p[2], p[4]);
    const V s1 = vadd(p[5], p[7]), s2 = vadd(p[6], p[8]);
    const V sd = vadd(s1, s2);
    const V base = vfma(Ln::set(-8.f), p[0], sd);
    const V m2xx = vfma(four, sx, vfma(Ln::set(-2.f), sy, base));
    const V m2yy = vfma(four, sy, vfma(Ln::set(-2.f), sx, base));
    const V m2xy = vmul(Ln::set(1.5f), vsub(s1, s2));
    const V tr = C.m2v ? vfma(Ln::set(-20.f), p[0], vfma(four, vadd(sx, sy), sd))
                       : vadd(m2xx, m2yy);
    const V ax = vfma(m1x, m2xx, vmul(m1y, m2xy));
    const V ay = vfma(m1x, m2xy, vmul(m1y, m2yy));
    const V cp = vfma(Ln::set(C.fsc), p[0], vmul(Ln::set(C.fk2), tr));
    const V kd = Ln::set(C.fkd);
    Fx = vfma(m1x, cp, vmul(kd, ax));
    Fy = vfma(m1y, cp, vmul(kd, ay));
}

__device__ __forceinline__ SiteConsts site_consts(const LatDev& L) {
    return SiteConsts{L.rho0, L.om1, L.rw0, L.rg0, L.ra, L.rd, L.ga9, L.gd9,
                      L.omega, L.guo, L.fsc, L.fk2, L.fkd, L.m2_variant, L.zero};
}

// ---- the stored outputs of a collision ----------------------------------------
// From Y0 = f*_0 - w_0 rho0 - r0 (the change of the rest deviation, small)
// and H_i = (f*_i - w_i rho0) - c'_i (f*_0 - w_0 rho0) (small), the nine
// values to store: R* = r0 + Y0 as the storage will hold it, and
// G*_i = H_i + E/8 with E = 9/4 (r0 - R*) + D - sum_i H_i, so that
// 9/4 R* + sum_i G*_i = 9/4 r0 + D: the site's pulled mass, which the
// collision conserves, up to the roundings of the small G*_i.
template <class S, class V>
__device__ __forceinline__ void rest_finish(const Site<V>& st, V Y0, const V H[9], V o[9]) {
    using Ln = Lanes<V>;
    V R = vadd(st.r0, Y0);
#pragma unroll
    for (int k = 0; k < Ln::n; ++k) Ln::put(R, k, S::rt(Ln::get(R, k)));
    const V sH = vadd(vadd(vadd(H[1], H[2]), vadd(H[3], H[4])), vadd(vadd(H[5], H[6]), vadd(H[7], H[8])));
    const V E = vfma(Ln::set(2.25f), vsub(st.r0, R), vsub(st.D, sH));
    o[0] = R;
#pragma unroll
    for (int i = 1; i < 9; ++i) o[i] = vfma(Ln::set(0.125f), E, H[i]);
}

// t / 3 correctly rounded (for all but rare ties): the rounded quotient,
// its exact remainder by an FMA, and one correction (the classic
// division-by-a-constant step, Muller et al., Handbook of Floating-Point
// Arithmetic).  Multiplying by the FP32 value of 1/3 instead would scale
// every quotient by the same 1 + 3e-8.
template <class V>
__device__ __forceinline__ V div3(V t) {
    using Ln = Lanes<V>;
    const V k = Ln::set(1.f / 3.f);
    const V q = vmul(t, k);
    return vfma(vfma(Ln::set(-3.f), q, t), k, q);
}

// ---- BGK collision with Guo forcing -------------------------------------------
// The pulled site in, the nine values to store out (rest_finish).
//   rho, j     Eqs. (FD), (FMD);  u = (j + F/2)/rho
//   f*_i = f_i - omega (f_i - f^eq_i) + (1 - 1/2tau) S_i       Eqs. (BGKCO), (GFSBGK)
//   f^eq_i - w_i rho0 = w_i (drho + rho (3 cu + 9/2 cu^2 - 3/2 u^2))   Eq. (SEDF)
//   S_i = w_i (3 cF + 9 cF cu - 3 F.u)                          Eq. (GFS)
// In the stored form the isotropic parts w_i (drho - 3/2 rho u^2) and
// -3 w_i F.u of f^eq_i and S_i cancel against c'_i times those of the rest
// population (c'_i w_0 = w_i), so for a pair of opposite directions c, -c
// of weight w
//   H_{+-} = (1 - omega) h_{+-} + cu (9/2 omega w rho cu + 9 guo w cF) +- Q,
//   Q = 3 w (omega rho cu + guo cF),
// and for the rest population (drho = 9/4 r0 + D, omega w_0 9/4 r0 = omega r0)
//   Y0 = w_0 (omega (D - 3/2 rho u^2) - 3 guo F.u).
// The odd parts Q carry the momentum, sum_i c_i f*_i = (1 - omega) j +
// omega rho u + guo F = j + F: they are formed as exact-constant products
// divided by 3 with correct rounding on the axes, and on the diagonals as
// (Q_x +- Q_y)/4 (3 w_d (omega rho cu_d + guo cF_d) with cu_d = u_x +- u_y),
// so no FP32 constant biases the momentum every step.  The even parts use
// 9/2 omega w and 9 guo w, exact in FP32 (omega/2, guo, ...).  Nothing is
// formed as a difference of two large numbers.
template <class S, class V>
__device__ __forceinline__ void collide_bgk(const SiteConsts& C, const Site<V>& st, const V p[9],
                                            V o[9]) {
    using Ln = Lanes<V>;
    const V* h = st.h;
    const V rho = site_rho(st, C.rho0);
    const V jx = vadd(vadd(vsub(h[1], h[3]), vsub(h[5], h[6])), vsub(h[8], h[7]));
    const V jy = vsub(vadd(vsub(h[2], h[4]), vadd(h[5], h[6])), vadd(h[7], h[8]));
    V Fx, Fy;
    site_force(C, p, Fx, Fy);
    const V inv = vrcp(rho);
    const V half = Ln::set(0.5f);
    const V ux = vmul(vfma(half, Fx, jx), inv);  // Eq. (FMD)
    const V uy = vmul(vfma(half, Fy, jy), inv);
    const V usq = vfma(ux, ux, vmul(uy, uy));
    const V Fu = vfma(Fx, ux, vmul(Fy, uy));
    const V Ra = vmul(Ln::set(C.ra), rho), Rd = vmul(Ln::set(C.rd), rho);
    const V Or = vmul(Ln::set(C.omega), rho);
    const V gu = Ln::set(C.guo), q4 = Ln::set(0.25f);
    const V om1 = Ln::set(C.om1);
    // odd parts: axes, then diagonals from them
    const V Qx = div3(vfma(Or, ux, vmul(gu, Fx)));
    const V Qy = div3(vfma(Or, uy, vmul(gu, Fy)));
    const V Q5 = vmul(q4, vadd(Qx, Qy)), Q6 = vmul(q4, vsub(Qy, Qx));
    V H[9];
#define PPLBM_PAIR(I, J, CU, CF, R, G9, QQ)                                \
    {                                                                      \
        const V cu = (CU), cF = (CF);                                      \
        const V z = vfma(R, cu, vmul(Ln::set(G9), cF));                    \
        const V ev = vmul(cu, z);                                          \
        H[I] = vadd(vfma(om1, h[I], ev), QQ);                              \
        H[J] = vsub(vfma(om1, h[J], ev), QQ);                              \
    }
    PPLBM_PAIR(1, 3, ux, Fx, Ra, C.ga9, Qx)
    PPLBM_PAIR(2, 4, uy, Fy, Ra, C.ga9, Qy)
    // the diagonal projections u.c = (j.c + F.c/2)/rho are products of their
    // own: no product ever feeds a paired add (see Eos<EOS_DF>)
    {
        const V F5 = vadd(Fx, Fy), F6 = vsub(Fy, Fx);
        const V cu5 = vmul(vfma(half, F5, vadd(jx, jy)), inv);
        const V cu6 = vmul(vfma(half, F6, vsub(jy, jx)), inv);
        PPLBM_PAIR(5, 7, cu5, F5, Rd, C.gd9, Q5)
        PPLBM_PAIR(6, 8, cu6, F6, Rd, C.gd9, Q6)
    }
#undef PPLBM_PAIR
    const V Y0 = vfma(Ln::set(C.rw0), vfma(vmul(Ln::set(-1.5f), rho), usq, st.D),
                      vmul(Ln::set(C.rg0), Fu));
    rest_finish<S>(st, Y0, H, o);
}

// MRT collision (Eq. MRTCO) with Guo forcing in moment space (Eq. GFSMRT),
// for the Gram-Schmidt matrix M of Appendix A.  Written on the
// non-equilibrium part n = f - f^eq, which is small, so rounding scales with
// it and not with rho:
//   f* = f^eq + M^-1 [ (I - Lambda) M n + (I - Lambda/2) M S ],
// the same update as f - M^-1 Lambda M (f - f^eq) + M^-1 (I - Lambda/2) M S.
// f^eq is the equilibrium of Eq. (SEDF); M S is the vector printed in
// Appendix A; the conserved moments of n are exact: (M n)_0 = 0,
// (M n)_3 = -F_x/2, (M n)_5 = -F_y/2 (Eq. FMD).  Back to populations with
// M^-1 = M^T D^-1, D = diag(9, 36, 36, 6, 12, 6, 12, 4, 4) (the rows of M are
// orthogonal).
// Everything is taken relative to c'_i r0 (r0 the pulled rest deviation):
// e_i = f^eq_i - w_i rho0 - c'_i r0 = w_i (base + rho (+-3 cu + 9/2 cu^2)) with
// base = D - 3/2 rho u^2 (drho = 9/4 r0 + D), n_i = h_i - e_i, n_0 = -e_0, and
// the update gives o_i = f*_i - w_i rho0 - c'_i r0, all small; the rest
// population's o_0 follows from mass conservation (sum_i o_i = D), and
// H_i = o_i - c'_i o_0 goes to rest_finish with Y0 = o_0.
// The sites are held in the lanes of V (paired FP32 for two sites), and the
// code follows the rule of the paired arithmetic: a product
// that is added enters an FMA, and a product needed as a value of its own
// (the equilibria) is an FMA with the zero addend the compiler cannot see.
// Two terms are simplified exactly: (1 - s3)(-Fx/2) + (1 - s3/2) Fx = Fx/2,
// and likewise Fy/2 for the fifth moment.
template <class S, class V>
__device__ __forceinline__ void collide_mrt(const SiteConsts& C, const float* s, const Site<V>& st,
                                            const V p[9], V o[9]) {
    using Ln = Lanes<V>;
    const V* h = st.h;
    const V z0 = Ln::set(C.zero), half = Ln::set(0.5f), mone = Ln::set(-1.f);
    const V rho = site_rho(st, C.rho0);
    const V jx = vadd(vadd(vsub(h[1], h[3]), vsub(h[5], h[6])), vsub(h[8], h[7]));
    const V jy = vsub(vadd(vsub(h[2], h[4]), vadd(h[5], h[6])), vadd(h[7], h[8]));
    V Fx, Fy;
    site_force(C, p, Fx, Fy);
    const V inv = vrcp(rho);
    const V ux = vmul(vfma(half, Fx, jx), inv);  // Eq. (FMD)
    const V uy = vmul(vfma(half, Fy, jy), inv);
    const V usq = vfma(ux, ux, vmul(uy, uy));
    const V uF = vfma(ux, Fx, vmul(uy, Fy));
    const V base = vfma(vmul(Ln::set(-1.5f), rho), usq, st.D);
    // equilibria relative to c'_i r0: w_i (base + 9/2 rho cu^2 +- 3 rho cu)
    const V r45 = vmul(Ln::set(4.5f), rho), r3 = vmul(Ln::set(3.f), rho);
    const V nr3 = vmul(Ln::set(-3.f), rho);
    V e[9];
    auto pair = [&](V cu, float w, int ip, int im) {
        const V t = vfma(vmul(r45, cu), cu, base);
        e[ip] = vfma(Ln::set(w), vfma(r3, cu, t), z0);
        e[im] = vfma(Ln::set(w), vfma(nr3, cu, t), z0);
    };
    pair(ux, 1.f / 9.f, 1, 3);
    pair(uy, 1.f / 9.f, 2, 4);
    pair(vadd(ux, uy), 1.f / 36.f, 5, 7);
    pair(vsub(uy, ux), 1.f / 36.f, 6, 8);
    e[0] = vfma(Ln::set(4.f / 9.f), base, z0);
    V n[9];
    n[0] = vmul(e[0], mone);
#pragma unroll
    for (int i = 1; i < 9; ++i) n[i] = vsub(h[i], e[i]);
    // non-conserved moments of n
    const V sa = vadd(vadd(n[1], n[2]), vadd(n[3], n[4]));
    const V sd = vadd(vadd(n[5], n[6]), vadd(n[7], n[8]));
    const V m1 = vfma(Ln::set(-4.f), n[0], vfma(Ln::set(2.f), sd, vmul(sa, mone)));
    const V m2 = vfma(Ln::set(4.f), n[0], vfma(Ln::set(-2.f), sa, sd));
    const V m4 = vfma(Ln::set(-2.f), n[1],
                      vfma(Ln::set(2.f), n[3], vadd(vsub(n[5], n[6]), vsub(n[8], n[7]))));
    const V m6 = vfma(Ln::set(-2.f), n[2],
                      vfma(Ln::set(2.f), n[4], vsub(vadd(n[5], n[6]), vadd(n[7], n[8]))));
    const V m7 = vadd(vsub(n[1], n[2]), vsub(n[3], n[4]));
    const V m8 = vadd(vsub(n[5], n[6]), vsub(n[7], n[8]));
    // (I - Lambda) M n + (I - Lambda/2) M S, moment by moment
    auto A = [&](int k) { return Ln::set(1.f - s[k]); };
    auto B = [&](int k, float f) { return Ln::set(f * (1.f - 0.5f * s[k])); };
    const V p1 = vfma(A(1), m1, vmul(B(1, 6.f), uF));
    const V p2 = vfma(A(2), m2, vmul(B(2, -6.f), uF));
    const V p3 = vmul(half, Fx);
    const V p4 = vfma(A(4), m4, vmul(B(4, -1.f), Fx));
    const V p5 = vmul(half, Fy);
    const V p6 = vfma(A(6), m6, vmul(B(6, -1.f), Fy));
    const V p7 = vfma(A(7), m7, vmul(B(7, 2.f), vfma(ux, Fx, vmul(vmul(uy, mone), Fy))));
    const V p8 = vfma(A(8), m8, vmul(B(8, 1.f), vfma(ux, Fy, vmul(uy, Fx))));
    // M^T D^-1 (the mass moment of the update is zero), with the 1/36, 1/6,
    // 1/12 and 1/4 of D^-1 and the entries of M as FMA multiplicands
    auto K = [](float c) { return Ln::set(c); };
    const V ax = vfma(p1, K(-1.f / 36.f), vmul(p2, K(-2.f / 36.f)));  // axis directions
    const V dg = vfma(p1, K(2.f / 36.f), vmul(p2, K(1.f / 36.f)));    // diagonals
    V q[9];
    q[1] = vfma(p3, K(1.f / 6.f), vfma(p4, K(-2.f / 12.f), vfma(p7, K(0.25f), vadd(e[1], ax))));
    q[2] = vfma(p5, K(1.f / 6.f), vfma(p6, K(-2.f / 12.f), vfma(p7, K(-0.25f), vadd(e[2], ax))));
    q[3] = vfma(p3, K(-1.f / 6.f), vfma(p4, K(2.f / 12.f), vfma(p7, K(0.25f), vadd(e[3], ax))));
    q[4] = vfma(p5, K(-1.f / 6.f), vfma(p6, K(2.f / 12.f), vfma(p7, K(-0.25f), vadd(e[4], ax))));
    // diagonals: e + dg +- (q3 + q4) +- (q5 + q6) +- q8
    const V d3 = vfma(p3, K(1.f / 6.f), vmul(p4, K(1.f / 12.f)));  // q3 + q4
    const V d5 = vfma(p5, K(1.f / 6.f), vmul(p6, K(1.f / 12.f)));  // q5 + q6
    q[5] = vfma(p8, K(0.25f), vadd(vadd(e[5], dg), vadd(d3, d5)));
    q[6] = vfma(p8, K(-0.25f), vadd(vadd(e[6], dg), vsub(d5, d3)));
    q[7] = vfma(p8, K(0.25f), vsub(vadd(e[7], dg), vadd(d3, d5)));
    q[8] = vfma(p8, K(-0.25f), vadd(vadd(e[8], dg), vsub(d3, d5)));
    const V Y0 = vsub(st.D, vadd(vadd(vadd(q[1], q[2]), vadd(q[3], q[4])),
                                 vadd(vadd(q[5], q[6]), vadd(q[7], q[8]))));
    V H[9];
#pragma unroll
    for (int i = 1; i < 9; ++i) H[i] = vfma(Ln::set(-cref(i)), Y0, q[i]);
    rest_finish<S>(st, Y0, H, o);
}

// One collision (BGK or MRT) of the sites held in the lanes of V.
template <class S, bool MRT, class V>
__device__ __forceinline__ void collide(const SiteConsts& C, const float* mrt_s, const Site<V>& st,
                                        const V p[9], V o[9]) {
    if (!MRT)
        collide_bgk<S>(C, st, p, o);
    else
        collide_mrt<S>(C, mrt_s, st, p, o);
}

// The periodic images of population i of site (x, y) that a step reads,
// without the site itself (which a bulk tile store writes).  Readers pull
// f*_i(x - c_i) for cells x from -1 to n: the single pass rebuilds psi on a
// one-site ring around each tile, the other passes pull for x in 0 .. n - 1
// only.  And every cell reads the rest plane at x - c for each c.  So along
// one axis, the image at x + n of a site x < GW (the high side) is read for
// c_i <= -x, the image at x - n of a site x >= n - GW (the low side) for
// c_i >= n - 1 - x, and the rest plane at every image.  With i a constant
// (an unrolled loop over the planes) the tests fold: a left-edge site skips
// the images of the planes that move to the left, and so on.  i = 0 (the
// rest plane) writes every image.
template <class T>
__device__ __forceinline__ void store_images(T* plane, int i, int pitch, int gx, int x, int y,
                                             int nx, int ny, T v) {
    T* const row = plane + (int64_t)(y + GY) * pitch + gx;
    const int cx = plane_cx(i), cy = plane_cy(i);
    const bool all = i == 0;
    const bool xl = x < GW && (all || cx <= -x), xh = x >= nx - GW && (all || cx >= nx - 1 - x);
    const bool yl = y < GW && (all || cy <= -y), yh = y >= ny - GW && (all || cy >= ny - 1 - y);
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

// Store the nine outputs of site (x, y): interior sites with plain stores,
// sites within GW of an edge also into all their periodic images.  `tile_in`
// says the whole tile is interior (uniform per block), which skips the
// per-site test.
template <class S>
__device__ __forceinline__ void store_site(typename S::T* o, int64_t plane, int pitch, int gx,
                                           int x, int y, int nx, int ny, const float v[9],
                                           bool tile_in = false) {
    if (tile_in || ((x >= GW) & (x < nx - GW) & (y >= GW) & (y < ny - GW))) {
        typename S::T* q = o + (int64_t)(y + GY) * pitch + (x + gx);
#pragma unroll
        for (int i = 0; i < 9; ++i) q[i * plane] = S::cv(v[i]);
    } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) store_img(o + i * plane, pitch, gx, x, y, nx, ny, S::cv(v[i]));
    }
}

// store_site writing only the periodic images a step reads (store_images):
// the batch form of the single pass, whose small lattices make edge sites
// common.  (Kept apart from store_site: the single-lattice kernel, which
// compiles store_site for its ragged tiles, ran 2 % slower with this form
// in it, measured.)
template <class S>
__device__ __forceinline__ void store_site_read(typename S::T* o, int64_t plane, int pitch, int gx,
                                                int x, int y, int nx, int ny, const float v[9],
                                                bool tile_in = false) {
    typename S::T* q = o + (int64_t)(y + GY) * pitch + (x + gx);
#pragma unroll
    for (int i = 0; i < 9; ++i) q[i * plane] = S::cv(v[i]);
    if (!tile_in && !((x >= GW) & (x < nx - GW) & (y >= GW) & (y < ny - GW))) {
#pragma unroll
        for (int i = 0; i < 9; ++i)
            store_images(o + i * plane, i, pitch, gx, x, y, nx, ny, S::cv(v[i]));
    }
}

}  // namespace pplbm
