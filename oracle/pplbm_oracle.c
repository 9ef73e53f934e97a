/*
 * pplbm_oracle.c -- plain FP64 CPU oracle for one time step of the D2Q9
 * pseudopotential lattice Boltzmann method with the nearest-neighbour
 * "force approach" of Czelusniak et al. (arXiv 2003.07968).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header, table or constant
 * generator with the CUDA path.
 *
 * Everything is written the slow, obvious way: one site at a time, double
 * precision, push streaming into a separate array, periodic boundaries.
 * Each function names the equation of the paper it follows.
 *
 * Readings of the paper taken here (where it is silent, garbled or
 * ambiguous):
 *   - the Shan-Chen term of the A_ij tensor is printed without c_{i alpha};
 *     the brute-force path restores it so that it matches Eq. (SCF);
 *   - the velocity inside the Guo source term (Eq. GFS) is the same
 *     force-shifted velocity as in the equilibrium (Eq. FMD);
 *   - M2_{beta beta} defaults to the direct trace of Eq. (SOMED); the
 *     alternative 2 c_s^2 (M0 - psi) named after Eq. (DFTCST) is a flag;
 *   - T in Eq. (CSEOS) is the reduced temperature (T_c = 1 for the printed
 *     constants a, b, c).
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fopenmp -shared -fPIC
 * (-ffp-contract=off keeps x86-64 and aarch64 results bit-identical).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_OOM (-2)
#define ORC_ERR_NUMERIC (-4)

/* Parameters of one lattice.  Field order is mirrored by the ctypes
 * structure in oracle/__init__.py. */
typedef struct {
    double tau;      /* BGK relaxation time, Eq. (BGKCO)                    */
    double G;        /* interaction parameter, Eq. (DED)                    */
    double eps;      /* epsilon of Eq. (IFT)                                 */
    double sigma;    /* sigma of Eq. (IFT)                                   */
    double T;        /* reduced temperature in Eq. (CSEOS)                   */
    double eos_a, eos_b, eos_c, eos_k; /* constants of Eq. (CSEOS)          */
    int32_t m2_trace_variant; /* 0: direct trace, 1: 2 c_s^2 (M0 - psi)     */
    int32_t collision;        /* 0: BGK (Eq. BGKCO), 1: MRT (Eq. MRTCO)     */
    double mrt_rates[9];      /* diagonal of Lambda, Eq. (RelaxationMatrix) */
    int32_t eos_kind;         /* 0: Carnahan-Starling, Eq. (CSEOS); 1: van der Waals */
} orc_params;

/* D2Q9 velocity set, Eq. (VelocitySet), and weights (text after Eq. SEDF). */
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double W[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                            1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                            1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
#define CS2 (1.0 / 3.0)

static int wrap(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}

/* The equation of state P_EOS(rho) that Eq. (DED) turns into psi:
 *   eos_kind 0, Carnahan-Starling, Eq. (CSEOS):
 *     P = k [c rho T (1 + b rho + (b rho)^2 - (b rho)^3) / (1 - b rho)^3 - a rho^2];
 *   eos_kind 1, van der Waals (the textbook form, in the same constants):
 *     P = k [c rho T / (1 - b rho) - a rho^2];
 *     with a = 3, b = 1/3, c = 8/3 it is the reduced equation
 *     P / k = 8 rho T / (3 - rho) - 3 rho^2, critical point (1, 1, k). */
double orc_eos_pressure(const orc_params* p, double rho) {
    double br = p->eos_b * rho;
    if (p->eos_kind == 1) return p->eos_k * (p->eos_c * rho * p->T / (1.0 - br) - p->eos_a * rho * rho);
    double num = 1.0 + br + br * br - br * br * br;
    double den = (1.0 - br) * (1.0 - br) * (1.0 - br);
    return p->eos_k * (p->eos_c * rho * p->T * num / den - p->eos_a * rho * rho);
}

/* Pseudopotential psi = sqrt((P_EOS - c_s^2 rho) / G), Eq. (DED).
 * Returns 0 and writes psi, or ORC_ERR_NUMERIC when rho is not positive and
 * finite, b*rho >= 1, or the radicand is negative. */
int orc_psi(const orc_params* p, double rho, double* psi) {
    if (!(rho > 0.0) || !isfinite(rho) || p->eos_b * rho >= 1.0) return ORC_ERR_NUMERIC;
    double arg = (orc_eos_pressure(p, rho) - CS2 * rho) / p->G;
    if (!(arg >= 0.0) || !isfinite(arg)) return ORC_ERR_NUMERIC;
    *psi = sqrt(arg);
    return ORC_OK;
}

/* psi over a whole field; returns the number of invalid sites (psi=NaN). */
int64_t orc_psi_field(const orc_params* p, int64_t n, const double* rho, double* psi) {
    int64_t bad = 0;
    for (int64_t s = 0; s < n; ++s) {
        if (orc_psi(p, rho[s], &psi[s]) != ORC_OK) {
            psi[s] = NAN;
            ++bad;
        }
    }
    return bad;
}

/* Force at one site from the nine values psi(x + c_i).
 * Moments of psi: Eqs. (ZOMED), (FOMED), (SOMED).
 * Discrete force terms: Eqs. (DFTCCC), (DFTCST).
 * Shan-Chen force: Eq. (SCF).  Combined force: Eq. (IFT). */
static void force_from_stencil(const orc_params* p, const double ps[9], double* Fx,
                               double* Fy) {
    double M0 = 0.0, M1x = 0.0, M1y = 0.0, M2xx = 0.0, M2yy = 0.0, M2xy = 0.0;
    for (int i = 0; i < 9; ++i) {
        double cx = CX[i], cy = CY[i];
        M0 += W[i] * ps[i];
        M1x += W[i] * cx * ps[i];
        M1y += W[i] * cy * ps[i];
        M2xx += W[i] * (cx * cx - CS2) * ps[i];
        M2yy += W[i] * (cy * cy - CS2) * ps[i];
        M2xy += W[i] * (cx * cy) * ps[i];
    }
    double cs4 = CS2 * CS2, cs6 = cs4 * CS2;
    double G = p->G;
    /* Eq. (SCF): F^SC = -psi(x) (2G/c_s^2) sum_i w_i psi(x+c_i) c_i = -psi (2G/c_s^2) M1 */
    double fscx = -ps[0] * (2.0 * G / CS2) * M1x;
    double fscy = -ps[0] * (2.0 * G / CS2) * M1y;
    /* M1_beta M2_{alpha beta} */
    double m1m2x = M1x * M2xx + M1y * M2xy;
    double m1m2y = M1x * M2xy + M1y * M2yy;
    /* Eq. (DFTCCC) */
    double f1x = -2.0 * m1m2x / cs6;
    double f1y = -2.0 * m1m2y / cs6;
    /* trace M2_{beta beta}: direct, or 2 c_s^2 (M0 - psi) */
    double tr = (p->m2_trace_variant == 1) ? 2.0 * CS2 * (M0 - ps[0]) : (M2xx + M2yy);
    /* Eq. (DFTCST) */
    double f2x = (M1x * tr - m1m2x) / cs6;
    double f2y = (M1y * tr - m1m2y) / cs6;
    /* Eq. (IFT) */
    *Fx = fscx - 0.75 * p->eps * CS2 * G * f1x + (p->sigma - 1.0) * CS2 * G * f2x;
    *Fy = fscy - 0.75 * p->eps * CS2 * G * f1y + (p->sigma - 1.0) * CS2 * G * f2y;
}

static void gather_stencil(int nx, int ny, const double* psi, int x, int y, double ps[9]) {
    for (int i = 0; i < 9; ++i)
        ps[i] = psi[(int64_t)wrap(y + CY[i], ny) * nx + wrap(x + CX[i], nx)];
}

/* Force field from a psi field through the moments (periodic lattice). */
void orc_force_moments(const orc_params* p, int nx, int ny, const double* psi, double* Fx,
                       double* Fy) {
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            double ps[9];
            gather_stencil(nx, ny, psi, x, y, ps);
            force_from_stencil(p, ps, &Fx[(int64_t)y * nx + x], &Fy[(int64_t)y * nx + x]);
        }
    }
}

/* The tensor A_ij of Eq. (Ansatz), written out after Eq. (PTIF)'s
 * derivation (printed just before Eq. PTIF), with the Shan-Chen term carrying
 * c_{i alpha} as Eq. (SCF) requires. */
static double a_tensor(const orc_params* p, int i, int j, int alpha) {
    double cs4 = CS2 * CS2;
    double G = p->G;
    double cia = alpha == 0 ? CX[i] : CY[i];
    double cja = alpha == 0 ? CX[j] : CY[j];
    double a = 0.0;
    if (j == 0) a += -(2.0 * G / CS2) * W[i] * cia;
    /* c_{i beta} (c_{j alpha} c_{j beta} - c_s^2 delta_{alpha beta}) */
    double t1 = 0.0;
    for (int beta = 0; beta < 2; ++beta) {
        double cib = beta == 0 ? CX[i] : CY[i];
        double cjb = beta == 0 ? CX[j] : CY[j];
        t1 += cib * (cja * cjb - CS2 * (alpha == beta ? 1.0 : 0.0));
    }
    /* c_{i alpha} (c_{j beta} c_{j beta} - c_s^2 delta_{beta beta}), delta_bb = 2 */
    double cj2 = (double)(CX[j] * CX[j] + CY[j] * CY[j]);
    double t2 = cia * (cj2 - CS2 * 2.0);
    double wij = (W[i] / CS2) * (W[j] / cs4);
    a += (1.5 * p->eps - (p->sigma - 1.0)) * CS2 * G * wij * t1;
    a += (p->sigma - 1.0) * CS2 * G * wij * t2;
    return a;
}

/* Force field as F_alpha = sum_i sum_j A_ij psi_i psi_j, Eq. (Ansatz).
 * Independent of the moment path; direct-trace reading only. */
void orc_force_brute(const orc_params* p, int nx, int ny, const double* psi, double* Fx,
                     double* Fy) {
    double A[2][9][9];
    for (int alpha = 0; alpha < 2; ++alpha)
        for (int i = 0; i < 9; ++i)
            for (int j = 0; j < 9; ++j) A[alpha][i][j] = a_tensor(p, i, j, alpha);
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            double ps[9];
            gather_stencil(nx, ny, psi, x, y, ps);
            double fx = 0.0, fy = 0.0;
            for (int i = 0; i < 9; ++i)
                for (int j = 0; j < 9; ++j) {
                    fx += A[0][i][j] * ps[i] * ps[j];
                    fy += A[1][i][j] * ps[i] * ps[j];
                }
            Fx[(int64_t)y * nx + x] = fx;
            Fy[(int64_t)y * nx + x] = fy;
        }
    }
}

/* Equilibrium distribution, Eq. (SEDF). */
static void equilibrium(double rho, double ux, double uy, double feq[9]) {
    double cs4 = CS2 * CS2;
    for (int i = 0; i < 9; ++i) {
        double cx = CX[i], cy = CY[i];
        double cu = cx * ux + cy * uy;
        double quad = (cx * cx - CS2) * ux * ux + 2.0 * cx * cy * ux * uy + (cy * cy - CS2) * uy * uy;
        feq[i] = W[i] * (rho + cu * rho / CS2 + quad * rho / (2.0 * cs4));
    }
}

/* Guo source term before the collision-dependent factor C_ij, Eq. (GFS):
 * w_i (c_i.F / c_s^2 + (c_ia c_ib - c_s^2 d_ab) F_a u_b / c_s^4). */
static void guo_raw(double Fx, double Fy, double ux, double uy, double s[9]) {
    double cs4 = CS2 * CS2;
    for (int i = 0; i < 9; ++i) {
        double cx = CX[i], cy = CY[i];
        double cF = cx * Fx + cy * Fy;
        double quad = (cx * cx - CS2) * Fx * ux + cx * cy * (Fx * uy + Fy * ux) + (cy * cy - CS2) * Fy * uy;
        s[i] = W[i] * (cF / CS2 + quad / cs4);
    }
}

/* Gram-Schmidt moment matrix, Eq. (MatrixMRT). */
static const double MRT_M[9][9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},
    {-4, -1, -1, -1, -1, 2, 2, 2, 2},
    {4, -2, -2, -2, -2, 1, 1, 1, 1},
    {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, -2, 0, 2, 0, 1, -1, -1, 1},
    {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {0, 0, -2, 0, 2, 1, 1, -1, -1},
    {0, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 1, -1, 1, -1},
};

/* Inverse of MRT_M by Gauss-Jordan elimination with partial pivoting. */
static void mrt_inverse(double inv[9][9]) {
    double a[9][18];
    for (int r = 0; r < 9; ++r)
        for (int c = 0; c < 18; ++c) a[r][c] = c < 9 ? MRT_M[r][c] : (c - 9 == r ? 1.0 : 0.0);
    for (int c = 0; c < 9; ++c) {
        int piv = c;
        for (int r = c + 1; r < 9; ++r)
            if (fabs(a[r][c]) > fabs(a[piv][c])) piv = r;
        if (piv != c)
            for (int k = 0; k < 18; ++k) {
                double t = a[c][k];
                a[c][k] = a[piv][k];
                a[piv][k] = t;
            }
        double d = a[c][c];
        for (int k = 0; k < 18; ++k) a[c][k] /= d;
        for (int r = 0; r < 9; ++r) {
            if (r == c) continue;
            double m = a[r][c];
            if (m == 0.0) continue;
            for (int k = 0; k < 18; ++k) a[r][k] -= m * a[c][k];
        }
    }
    for (int r = 0; r < 9; ++r)
        for (int c = 0; c < 9; ++c) inv[r][c] = a[r][c + 9];
}

/* Post-collision populations at one site.
 * BGK: f* = f - (f - feq)/tau + (1 - 1/(2 tau)) s, Eqs. (TLBE), (BGKCO), (GFSBGK).
 * MRT: f* = f - M^-1 Lambda M (f - feq) + M^-1 (I - Lambda/2) M s,
 *      Eqs. (MRTCO), (GFSMRT). */
static void collide_site(const orc_params* p, const double minv[9][9], const double f[9],
                         double rho, double ux, double uy, double Fx, double Fy, double out[9]) {
    double feq[9], s[9];
    equilibrium(rho, ux, uy, feq);
    guo_raw(Fx, Fy, ux, uy, s);
    if (p->collision == 0) {
        double c = 1.0 - 1.0 / (2.0 * p->tau);
        for (int i = 0; i < 9; ++i) out[i] = f[i] - (f[i] - feq[i]) / p->tau + c * s[i];
        return;
    }
    double mneq[9], ms[9];
    for (int r = 0; r < 9; ++r) {
        double a = 0.0, b = 0.0;
        for (int c = 0; c < 9; ++c) {
            a += MRT_M[r][c] * (f[c] - feq[c]);
            b += MRT_M[r][c] * s[c];
        }
        mneq[r] = p->mrt_rates[r] * a;
        ms[r] = (1.0 - 0.5 * p->mrt_rates[r]) * b;
    }
    for (int i = 0; i < 9; ++i) {
        double a = 0.0;
        for (int r = 0; r < 9; ++r) a += minv[i][r] * (ms[r] - mneq[r]);
        out[i] = f[i] + a;
    }
}

/* Equilibrium (Eq. SEDF) and raw Guo source (Eq. GFS without C_ij) at one
 * site, exposed so tests can compare their moments M f with the vectors the
 * paper prints in its MRT appendix. */
void orc_site_terms(double rho, double ux, double uy, double Fx, double Fy, double feq[9],
                    double s[9]) {
    equilibrium(rho, ux, uy, feq);
    guo_raw(Fx, Fy, ux, uy, s);
}

/* f = feq(rho, u) everywhere, the initialisation described after Eq. (ISD).
 * Layout of f: [9][ny][nx].  ux, uy may be NULL (zero velocity). */
void orc_init_equilibrium(int nx, int ny, const double* rho, const double* ux,
                          const double* uy, double* f) {
    int64_t n = (int64_t)nx * ny;
    for (int64_t s = 0; s < n; ++s) {
        double feq[9];
        equilibrium(rho[s], ux ? ux[s] : 0.0, uy ? uy[s] : 0.0, feq);
        for (int i = 0; i < 9; ++i) f[i * n + s] = feq[i];
    }
}

/* Density, Eq. (FD). */
static void density_field(int nx, int ny, const double* f, double* rho) {
    int64_t n = (int64_t)nx * ny;
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < n; ++s) {
        double r = 0.0;
        for (int i = 0; i < 9; ++i) r += f[i * n + s];
        rho[s] = r;
    }
}

static int64_t psi_field_checked(const orc_params* p, int64_t n, const double* rho, double* psi) {
    int64_t bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (int64_t s = 0; s < n; ++s) {
        if (orc_psi(p, rho[s], &psi[s]) != ORC_OK) {
            psi[s] = NAN;
            bad += 1;
        }
    }
    return bad;
}

/* Advance f (post-streaming populations, layout [9][ny][nx]) by nsteps time
 * steps of Eq. (TLBE) with push streaming on periodic boundaries.
 * Per step: rho (Eq. FD), psi (Eq. DED), force (Eq. IFT), velocity (Eq. FMD),
 * collision with Guo forcing, streaming f_i(x + c_i) <- f*_i(x).
 * Returns ORC_OK, or ORC_ERR_NUMERIC (psi undefined somewhere) with
 * *steps_done set to the number of completed steps. */
int orc_step(const orc_params* p, int nx, int ny, double* f, int64_t nsteps,
             int64_t* steps_done) {
    if (nx < 1 || ny < 1 || nsteps < 0) return ORC_ERR_ARG;
    int64_t n = (int64_t)nx * ny;
    double* rho = (double*)malloc(sizeof(double) * n);
    double* psi = (double*)malloc(sizeof(double) * n);
    double* fn = (double*)malloc(sizeof(double) * 9 * n);
    if (!rho || !psi || !fn) {
        free(rho);
        free(psi);
        free(fn);
        return ORC_ERR_OOM;
    }
    double minv[9][9];
    mrt_inverse(minv);
    int rc = ORC_OK;
    int64_t t = 0;
    for (; t < nsteps; ++t) {
        density_field(nx, ny, f, rho);
        if (psi_field_checked(p, n, rho, psi) != 0) {
            rc = ORC_ERR_NUMERIC;
            break;
        }
#pragma omp parallel for schedule(static)
        for (int y = 0; y < ny; ++y) {
            for (int x = 0; x < nx; ++x) {
                int64_t s = (int64_t)y * nx + x;
                double ps[9], fs[9], out[9], Fx, Fy;
                gather_stencil(nx, ny, psi, x, y, ps);
                force_from_stencil(p, ps, &Fx, &Fy);
                double r = 0.0, jx = 0.0, jy = 0.0;
                for (int i = 0; i < 9; ++i) {
                    fs[i] = f[i * n + s];
                    r += fs[i];
                    jx += fs[i] * CX[i];
                    jy += fs[i] * CY[i];
                }
                double ux = (jx + 0.5 * Fx) / r; /* Eq. (FMD) */
                double uy = (jy + 0.5 * Fy) / r;
                collide_site(p, minv, fs, r, ux, uy, Fx, Fy, out);
                for (int i = 0; i < 9; ++i) {
                    int xd = wrap(x + CX[i], nx), yd = wrap(y + CY[i], ny);
                    fn[i * n + (int64_t)yd * nx + xd] = out[i];
                }
            }
        }
        memcpy(f, fn, sizeof(double) * 9 * n);
    }
    if (steps_done) *steps_done = t;
    free(rho);
    free(psi);
    free(fn);
    return rc;
}

/* Macroscopic fields of the state f: rho (Eq. FD), force (Eq. IFT) from the
 * psi of this rho, and the force-shifted velocity (Eq. FMD).  Any output
 * pointer may be NULL. */
int orc_moments(const orc_params* p, int nx, int ny, const double* f, double* rho_out,
                double* ux, double* uy, double* Fx_out, double* Fy_out) {
    int64_t n = (int64_t)nx * ny;
    double* rho = (double*)malloc(sizeof(double) * n);
    double* psi = (double*)malloc(sizeof(double) * n);
    double* Fx = (double*)malloc(sizeof(double) * n);
    double* Fy = (double*)malloc(sizeof(double) * n);
    if (!rho || !psi || !Fx || !Fy) {
        free(rho);
        free(psi);
        free(Fx);
        free(Fy);
        return ORC_ERR_OOM;
    }
    density_field(nx, ny, f, rho);
    int rc = psi_field_checked(p, n, rho, psi) ? ORC_ERR_NUMERIC : ORC_OK;
    orc_force_moments(p, nx, ny, psi, Fx, Fy);
    for (int64_t s = 0; s < n; ++s) {
        double jx = 0.0, jy = 0.0;
        for (int i = 0; i < 9; ++i) {
            jx += f[i * n + s] * CX[i];
            jy += f[i * n + s] * CY[i];
        }
        if (rho_out) rho_out[s] = rho[s];
        if (ux) ux[s] = (jx + 0.5 * Fx[s]) / rho[s];
        if (uy) uy[s] = (jy + 0.5 * Fy[s]) / rho[s];
        if (Fx_out) Fx_out[s] = Fx[s];
        if (Fy_out) Fy_out[s] = Fy[s];
    }
    free(rho);
    free(psi);
    free(Fx);
    free(Fy);
    return rc;
}

/* Total mass sum_x sum_i f_i, in FP64, row sums added in row order so the
 * result does not depend on the thread count. */
double orc_mass(int nx, int ny, const double* f) {
    int64_t n = (int64_t)nx * ny;
    double* rows = (double*)malloc(sizeof(double) * ny);
    if (!rows) return NAN;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y) {
        double r = 0.0;
        for (int x = 0; x < nx; ++x)
            for (int i = 0; i < 9; ++i) r += f[i * n + (int64_t)y * nx + x];
        rows[y] = r;
    }
    double m = 0.0;
    for (int y = 0; y < ny; ++y) m += rows[y];
    free(rows);
    return m;
}

/* Number of OpenMP threads the oracle runs with (1 without OpenMP). */
int orc_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int n) {
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
