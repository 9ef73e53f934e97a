// lbm_layout.h -- per-lattice layout and constants (LatDev) from a lattice
// descriptor; shared by the handle runtime and the server.
#pragma once
#include <cmath>
#include <string>
#include <vector>

#include "../../include/pplbm.h"
#include "lbm_device.cuh"

namespace pplbm {

inline int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

inline void split_df(double v, df2& out) {
    out.hi = (float)v;
    out.lo = (float)(v - (double)out.hi);
}

// Everything of a lattice's LatDev except its offsets in the arenas:
// pitched planes with a ghost frame (16 bytes of columns and GY rows on each
// side), pitch a multiple of 32 bytes, planes multiples of 256 bytes, and
// the constants of the force (Eq. IFT), collision (Eqs. BGKCO, GFSBGK) and
// EOS (Eqs. DED, CSEOS).
inline LatDev lat_layout(const lbm_lattice_desc& d, int index) {
    LatDev L{};
    const int s = d.storage == LBM_STORE_F16_DEV ? 2 : 4;
    const int gx = 16 / s;
    L.nx = d.nx;
    L.ny = d.ny;
    L.gx = gx;
    L.pitch = (int)round_up(d.nx + 2 * gx, 32 / s);
    const int64_t rows = d.ny + 2 * GY;
    L.plane = round_up((int64_t)L.pitch * rows, 256 / s);
    L.gx_psi = 4;
    L.pitch_psi = (int)round_up(d.nx + 8, 8);
    // omega rounded once; 1 - omega, guo = 1 - omega/2 and the other BGK
    // constants but rw0, rg0 are exact FP32 functions of it, so that a
    // collision adds exactly F to the momentum in real arithmetic
    L.omega = (float)(1.0 / d.tau);
    L.guo = 1.f - 0.5f * L.omega;
    L.om1 = 1.f - L.omega;
    L.ra = 0.5f * L.omega;
    L.rd = 0.125f * L.omega;
    L.ga9 = L.guo;
    L.gd9 = 0.25f * L.guo;
    L.rw0 = (float)(4.0 * (double)L.omega / 9.0);
    L.rg0 = (float)(-3.0 * (double)L.guo * 4.0 / 9.0);
    // The force constant of the Shan-Chen term, -2G/c_s^2/36 = -G/6, rounded
    // to FP32, fixes the G the force acts with, Ge = -6 fsc; psi (Eq. DED)
    // and the other force terms are evaluated with that same Ge, so that
    // G psi^2 = P_EOS - c_s^2 rho holds for the force the kernels apply (a G
    // in psi that differs from the force's by the rounding of 1/6 would
    // shift the mechanical balance of an interface every step).
    L.fsc = (float)(-6.0 * d.G / 36.0);
    const double Ge = L.fsc != 0.f ? -6.0 * (double)L.fsc : d.G;
    L.k_sc = (float)(-6.0 * Ge);
    L.k1 = (float)(13.5 * d.eps * Ge);
    L.k2 = (float)(9.0 * (d.sigma - 1.0) * Ge);
    {
        const double k1 = 13.5 * d.eps * Ge, k2 = 9.0 * (d.sigma - 1.0) * Ge;
        L.fk2 = (float)(k2 / 1944.0);
        L.fkd = (float)((k1 - k2) / 1944.0);
    }
    L.rho0 = (d.storage == LBM_STORE_F32 || d.rho0 < 0.0) ? 0.f : (float)d.rho0;
    L.m2_variant = d.m2_trace_variant;
    L.eos_kind = d.eos_kind;
    L.lattice = index;
    L.row0 = -1;
    // psi^2 = rho (e1 q - e2 rho - e3): e1 = k c T / Ge, e2 = k a / Ge, e3 = 1/(3 Ge)
    L.eb = d.eos_b;
    L.e1 = d.eos_k * d.eos_c * d.T / Ge;
    L.e2 = d.eos_k * d.eos_a / Ge;
    L.e3 = 1.0 / (3.0 * Ge);
    split_df(L.eb, L.fb);
    split_df(L.e2, L.f2);
    split_df(L.e1 - L.e3, L.fc0);      // psi^2/rho = c0 + rho (C1 r^2 (1 + r) - e2)
    split_df((d.eos_kind == LBM_EOS_KIND_VDW ? 1.0 : 2.0) * L.eb * L.e1, L.fC1);
    L.sb = (float)L.eb;
    L.s1 = (float)L.e1;
    L.s2 = (float)L.e2;
    L.s3 = (float)L.e3;
    L.zero = 0.f;
    for (int i = 0; i < 9; ++i) L.mrt_s[i] = (float)d.mrt_rates[i];
    return L;
}

// Checks of one lattice descriptor (sizes, relaxation time, finite
// parameters, known enums).  Returns LBM_OK or LBM_ERR_ARG with `why`.
inline int validate_desc(const lbm_lattice_desc& d, std::string& why) {
    if (d.nx < 2 || d.ny < 2) return why = "nx and ny must be >= 2", LBM_ERR_ARG;
    if ((int64_t)d.nx * d.ny > (int64_t)1 << 31) return why = "lattice too large", LBM_ERR_ARG;
    if (!(d.tau > 0.5) || !std::isfinite(d.tau)) return why = "tau must be > 0.5", LBM_ERR_ARG;
    if (!(d.G != 0.0) || !std::isfinite(d.G)) return why = "G must be nonzero", LBM_ERR_ARG;
    if (!std::isfinite(d.eps) || !std::isfinite(d.sigma) || !std::isfinite(d.T) ||
        !std::isfinite(d.rho0) || d.rho0 > 1e6)
        return why = "non-finite parameter", LBM_ERR_ARG;
    if (!(d.eos_b > 0.0) || !std::isfinite(d.eos_a) || !std::isfinite(d.eos_c) ||
        !std::isfinite(d.eos_k))
        return why = "bad EOS constants", LBM_ERR_ARG;
    if (d.storage < LBM_STORE_F32 || d.storage > LBM_STORE_F16_DEV)
        return why = "unknown storage", LBM_ERR_ARG;
    if (d.eos_precision < LBM_EOS_F64 || d.eos_precision > LBM_EOS_F32)
        return why = "unknown eos_precision", LBM_ERR_ARG;
    if (d.m2_trace_variant != 0 && d.m2_trace_variant != 1)
        return why = "m2_trace_variant must be 0 or 1", LBM_ERR_ARG;
    if (d.collision != LBM_COLL_BGK && d.collision != LBM_COLL_MRT)
        return why = "unknown collision", LBM_ERR_ARG;
    if (d.eos_kind != LBM_EOS_KIND_CS && d.eos_kind != LBM_EOS_KIND_VDW)
        return why = "unknown eos_kind", LBM_ERR_ARG;
    if (d.collision == LBM_COLL_MRT)
        for (int i = 0; i < 9; ++i)
            if (!(d.mrt_rates[i] > 0.0 && d.mrt_rates[i] < 2.0))
                return why = "MRT rates must lie in (0, 2)", LBM_ERR_ARG;
    return LBM_OK;
}

// Per-pass defaults of LBM_KERNEL_AUTO for the plain-load kernels: psi pass
// 64 x 4 tiles, collision (or single) pass 32 x 8 tiles, both with two sites
// per thread.  (The single pass defaults to the TMA kernel with 32 x 16 tiles
// wherever the arena can be one tensor; see lbm_create.)
struct PassDefault {
    int variant, tx, ty, spt;
};
constexpr PassDefault kPassDefaults[2] = {{LBM_KERNEL_PLAIN, 64, 4, 2},
                                          {LBM_KERNEL_PLAIN, 32, 8, 2}};

// Automatic deviation reference: the smallest density of the field (not
// below 0), from field_scan's minimum.
inline float auto_rho0_of_min(double mn) { return (float)(mn > 0.0 ? mn : 0.0); }

// Row-space layout of a batch: every lattice with the same pitch P (the
// widest lattice's) and its nx + 2 GY rows stacked, lattice after lattice,
// inside each of the 18 planes (buffer A's nine, then B's), so that one 3-D
// tensor map (x: P, y: all rows, z: 18 planes) covers every lattice.  Sets
// pitch, plane, off_f and row0 of each lattice and returns the population
// elements of the arena; returns -1 (and changes nothing) when the common
// pitch would cost more than `max_waste` times the compact layout's memory.
inline int64_t row_space_layout(std::vector<LatDev>& lats, int es, double max_waste) {
    int P = 0;
    int64_t rows = 0, compact = 0;
    for (const LatDev& L : lats) {
        P = P > L.pitch ? P : L.pitch;
        rows += L.ny + 2 * GY;
        compact += 18 * L.plane;
    }
    const int64_t plane = round_up((int64_t)P * rows, 256 / es);
    if ((double)(18 * plane) > max_waste * (double)compact) return -1;
    int64_t r = 0;
    for (LatDev& L : lats) {
        L.pitch = P;
        L.plane = plane;
        L.row0 = (int32_t)r;
        L.off_f[0] = r * P;
        L.off_f[1] = L.off_f[0] + 9 * plane;
        r += L.ny + 2 * GY;
    }
    return 18 * plane;
}

// Elements of the two population buffers (A then B, nine planes each).
inline int64_t lat_pop_elems(const LatDev& L) { return 18 * L.plane; }
// Floats of the psi plane.
inline int64_t lat_psi_elems(const LatDev& L) {
    return round_up((int64_t)L.pitch_psi * (L.ny + 2 * GY), 64);
}

}  // namespace pplbm
