"""Host-side theory of arXiv 2003.07968, in plain numpy/scipy FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

* Carnahan-Starling EOS, Eq. (CSEOS), and psi, Eq. (DED); the van der Waals
  EOS in the same constants (kind="vdw") behind the same psi.
* Maxwell equal-area coexistence, Eq. (MLVDR) with equal bulk pressures.
* Mechanical-stability coexistence of the pseudopotential method,
  Eq. (PGLDR) with Eqs. (BPLP), (BPVP), epsilon = -2 A1 / (A2 + A3).
* Planar interface, Eqs. (PTNNPI), (PTTTPI), (STDIM), (STPI): density profile
  by central differences and Newton-Raphson, surface tension gamma_pi.
* Lamb's oscillation period, Eq. (DOP).
* Young-Laplace analysis of a static droplet, Eq. (YLR), with the interface
  at rho_m = (rho_l + rho_g)/2 (Sec. IV.B).
* Steady-state criterion, Eq. (SSC).
"""
from __future__ import annotations

import math
import warnings

import numpy as np
from scipy import integrate, optimize, sparse
from scipy.sparse import linalg as sparse_linalg

CS2 = 1.0 / 3.0
CS_A = 3.852462257
CS_B = 0.1304438842
CS_C = 2.785855166
CS_K = 0.01
VDW = (3.0, 1.0 / 3.0, 8.0 / 3.0, 0.01)  # reduced van der Waals, critical point (1, 1, k)
_CONST = {"cs": (CS_A, CS_B, CS_C, CS_K), "vdw": VDW}


def eos_pressure(rho, T, a=None, b=None, c=None, k=None, kind="cs"):
    """The equation of state of Eq. (DED).
    kind "cs", Eq. (CSEOS): P = k [c rho T (1 + b rho + (b rho)^2 - (b rho)^3)/(1 - b rho)^3 - a rho^2];
    kind "vdw": P = k [c rho T / (1 - b rho) - a rho^2] (van der Waals)."""
    A, B, C, K = _CONST[kind]
    a, b, c, k = (A if a is None else a, B if b is None else b, C if c is None else c,
                  K if k is None else k)
    br = b * rho
    if kind == "vdw":
        return k * (c * rho * T / (1 - br) - a * rho**2)
    return k * (c * rho * T * (1 + br + br**2 - br**3) / (1 - br) ** 3 - a * rho**2)


def dpdrho(rho, T, kind="cs"):
    """dP/drho by the complex-step derivative (exact to rounding for analytic P)."""
    h = 1e-30
    return np.imag(eos_pressure(np.asarray(rho, dtype=complex) + 1j * h, T, kind=kind)) / h


def psi(rho, T, G=-1.0, kind="cs"):
    """Eq. (DED): psi = sqrt((P_EOS - c_s^2 rho)/G)."""
    return np.sqrt((eos_pressure(rho, T, kind=kind) - CS2 * rho) / G)


def critical_point(a=None, b=None, c=None, k=None, kind="cs"):
    """(rho_c, T_c, P_c): where dP/drho = d2P/drho2 = 0 (plain root solve)."""

    def p(r, t):
        return eos_pressure(r, t, a, b, c, k, kind=kind)

    def d1(r, t):
        hc = 1e-30
        return np.imag(p(complex(r, hc), t)) / hc

    def eqs(v):
        r, t = v
        h = 1e-5
        return [d1(r, t) * 1e2, (d1(r + h, t) - d1(r - h, t)) / (2 * h) * 1e2]

    with warnings.catch_warnings():
        warnings.simplefilter("ignore", RuntimeWarning)
        r, t = optimize.fsolve(eqs, [0.9, 1.1], xtol=1e-14)
    return r, t, p(r, t)


def _spinodals(T, kind="cs"):
    """Densities where dP/drho = 0 (the van-der-Waals loop ends), T < 1."""
    b = _CONST[kind][1]
    rs = np.linspace(1e-3, 1 / b - 1e-3, 20001)
    d = dpdrho(rs, T, kind)
    idx = np.where(np.sign(d[:-1]) != np.sign(d[1:]))[0]
    roots = [optimize.brentq(lambda r: dpdrho(r, T, kind), rs[i], rs[i + 1], xtol=1e-15)
             for i in idx]
    if len(roots) < 2:
        raise ValueError(f"no two-phase region at T={T}")
    return roots[0], roots[1]


def maxwell(T, kind="cs"):
    """Maxwell coexistence (rho_g, rho_l) at reduced temperature T.

    Unknown p0 with P(rho_g) = P(rho_l) = p0 and the equal-area condition of
    Eq. (MLVDR), int_{rho_g}^{rho_l} (p0 - P) drho / rho^2 = 0.
    """
    s1, s2 = _spinodals(T, kind)
    pmin = eos_pressure(s2, T, kind=kind)
    pmax = eos_pressure(s1, T, kind=kind)
    b = _CONST[kind][1]

    def roots(p0):
        rg = optimize.brentq(lambda r: eos_pressure(r, T, kind=kind) - p0, 1e-12, s1, xtol=1e-15)
        rl = optimize.brentq(lambda r: eos_pressure(r, T, kind=kind) - p0, s2, 1 / b - 1e-9,
                             xtol=1e-15)
        return rg, rl

    def area(p0):
        rg, rl = roots(p0)
        val, _ = integrate.quad(lambda r: (p0 - eos_pressure(r, T, kind=kind)) / r**2, rg, rl,
                                epsabs=1e-15, epsrel=1e-13, limit=400)
        return val

    lo = max(pmin, 0.0) + 1e-9 * pmax
    p0 = optimize.brentq(area, lo, pmax * (1 - 1e-9), xtol=1e-17, rtol=1e-14)
    return roots(p0)


def pgldr(T, eps, G=-1.0, kind="cs"):
    """Coexistence (rho_g, rho_l) of the pseudopotential method, Eq. (PGLDR):
    int_{rho_g}^{rho_l} (p0 - c_s^2 rho - G psi^2) psidot / psi^(1+eps) drho = 0,
    with p0 = c_s^2 rho + G psi(rho)^2 at both ends (Eqs. BPLP, BPVP).  Since
    c_s^2 rho + G psi^2 = P_EOS by Eq. (DED), the bulk condition is
    P(rho_g) = P(rho_l) = p0.  psidot comes from 2 psi psidot = (P' - c_s^2)/G."""
    s1, s2 = _spinodals(T, kind)
    pmin = eos_pressure(s2, T, kind=kind)
    pmax = eos_pressure(s1, T, kind=kind)
    b = _CONST[kind][1]

    def roots(p0):
        rg = optimize.brentq(lambda r: eos_pressure(r, T, kind=kind) - p0, 1e-12, s1, xtol=1e-15)
        rl = optimize.brentq(lambda r: eos_pressure(r, T, kind=kind) - p0, s2, 1 / b - 1e-9,
                             xtol=1e-15)
        return rg, rl

    def integrand(r, p0):
        ps = psi(r, T, G, kind)
        # psidot from 2 psi psidot = (P' - c_s^2)/G
        psidot = (dpdrho(r, T, kind) - CS2) / (2 * G * ps)
        return (p0 - CS2 * r - G * ps**2) * psidot / ps ** (1 + eps)

    def area(p0):
        rg, rl = roots(p0)
        with warnings.catch_warnings():
            warnings.simplefilter("ignore", integrate.IntegrationWarning)
            val, _ = integrate.quad(integrand, rg, rl, args=(p0,), epsabs=1e-15,
                                    epsrel=1e-13, limit=400)
        return val

    lo = max(pmin, 0.0) + 1e-9 * pmax
    p0 = optimize.brentq(area, lo, pmax * (1 - 1e-9), xtol=1e-17, rtol=1e-14)
    return roots(p0)


def planar_interface(T, eps, sigma=1.0, L=30.0, dx=0.05, G=-1.0, max_newton=30):
    """Planar liquid-gas interface of the pressure tensor Eq. (GPTRF), Sec. II.

    The procedure the paper describes after Eq. (STPI):
      1. phase densities rho_g, rho_l from Eq. (PGLDR) (with Eqs. BPLP, BPVP),
         used as boundary values at x = 0 and x = L;
      2. mechanical equilibrium p_xx = p0 along x, Eq. (PTNNPI),
            c_s^2 rho + G psi^2 + G [A1 psi'^2 + (A2 + A3) psi psi''] = p0,
         with second-order central differences on a uniform mesh of spacing
         dx, solved by Newton-Raphson;
      3. psi(x) = psi(rho(x)), Eq. (DED);
      4. gamma_pi = int (p_xx - p_yy) dx, Eq. (STDIM), with Eqs. (PTNNPI),
         (PTTTPI): the integrand is G A3 psi psi'' (trapezoid rule, psi'' by
         central differences).
    Coefficients of the proposed force, Eq. (PTIFT): A1 = -3 eps c_s^2 / 4,
    A2 + A3 = 3 c_s^2 / 2, A3 = sigma c_s^2.

    Two readings.  Eq. (STPI) is printed as int A3 psi psi'' dx without G;
    p_xx - p_yy from Eqs. (PTNNPI), (PTTTPI) is G A3 psi psi'', which gives a
    positive gamma for G < 0, so G is kept.  With bulk densities at both
    ends the discrete problem is invariant, up to terms exponentially small
    in L, under translating the interface, so Newton steps along that mode
    are ill conditioned; the interface is pinned, rho = (rho_g + rho_l)/2 at
    the middle node, and p0 joins the unknowns (it converges to the p0 of
    Eq. PGLDR as L grows).

    Returns (x, rho, p0, gamma).
    """
    A1 = -0.75 * eps * CS2
    A23 = 1.5 * CS2
    A3 = sigma * CS2
    rho_g, rho_l = pgldr(T, eps, G)
    n = int(round(L / dx))
    if n < 4 or n % 2:
        raise ValueError("L / dx must be an even integer >= 4")
    x = np.arange(n + 1) * dx
    c = n // 2
    rho_m = 0.5 * (rho_g + rho_l)
    # initial profile: a tanh of width 2.5 centred at the pinned node
    rho = rho_m + 0.5 * (rho_l - rho_g) * np.tanh((x - x[c]) / 2.5)
    rho[0], rho[-1] = rho_g, rho_l
    p0 = float(eos_pressure(rho_g, T))
    m = n - 1  # interior unknowns rho_1 .. rho_{n-1}; unknown m is p0

    def psidot(r):
        # 2 psi psidot = (P' - c_s^2) / G
        return (dpdrho(r, T) - CS2) / (2 * G * psi(r, T, G))

    for _ in range(max_newton):
        ps = psi(rho, T, G)
        pd = psidot(rho)
        d1 = (ps[2:] - ps[:-2]) / (2 * dx)
        d2 = (ps[2:] - 2 * ps[1:-1] + ps[:-2]) / dx**2
        # c_s^2 rho + G psi^2 = P_EOS (Eq. DED)
        res = eos_pressure(rho[1:-1], T) + G * (A1 * d1**2 + A23 * ps[1:-1] * d2) - p0
        pin = rho[c] - rho_m
        # Jacobian: tridiagonal in rho, a column for p0 and the pin row
        sub = G * (-A1 * d1 / dx + A23 * ps[1:-1] / dx**2) * pd[:-2]
        sup = G * (A1 * d1 / dx + A23 * ps[1:-1] / dx**2) * pd[2:]
        dia = dpdrho(rho[1:-1], T) + G * A23 * (d2 - 2 * ps[1:-1] / dx**2) * pd[1:-1]
        J = sparse.lil_matrix((m + 1, m + 1))
        J.setdiag(dia)
        J.setdiag(sub[1:], -1)
        J.setdiag(sup[:-1], 1)
        J[:m, m] = -1.0
        J[m, c - 1] = 1.0
        step = sparse_linalg.spsolve(J.tocsc(), -np.r_[res, pin])
        rho[1:-1] += step[:m]
        p0 += step[m]
        if np.max(np.abs(step[:m])) < 1e-13 * rho_l:
            break
    ps = psi(rho, T, G)
    d2 = (ps[2:] - 2 * ps[1:-1] + ps[:-2]) / dx**2
    # the integrand vanishes in the bulk at both ends
    gamma = G * A3 * integrate.trapezoid(np.r_[0.0, ps[1:-1] * d2, 0.0], dx=dx)
    return x, rho, p0, float(gamma)


def lamb_period(gamma, rho_l, r_max, r_min, n=2):
    """Eq. (DOP): T_a = 2 pi [n (n^2 - 1) gamma / (rho_l R_m^3)]^(-1/2), R_m = sqrt(R_max R_min)."""
    rm = math.sqrt(r_max * r_min)
    return 2 * math.pi * (n * (n * n - 1) * gamma / (rho_l * rm**3)) ** -0.5


def steady_state_metric(rho_now, rho_before):
    """Left side of Eq. (SSC): sum|rho(t) - rho(t-100)| / sum|rho(t)|."""
    return float(np.abs(rho_now - rho_before).sum() / np.abs(rho_now).sum())


def droplet_radius(rho, rho_l, rho_g, center=None):
    """Radius where rho crosses rho_m = (rho_l + rho_g)/2 (Sec. IV.B), as the
    mean of the linearly interpolated crossings on the four axis rays from
    the centre node."""
    ny, nx = rho.shape
    cx, cy = (nx // 2, ny // 2) if center is None else center
    rm = 0.5 * (rho_l + rho_g)
    rays = [rho[cy, cx:], rho[cy, cx::-1], rho[cy:, cx], rho[cy::-1, cx]]
    rs = []
    for ray in rays:
        above = ray > rm
        k = int(np.argmin(above)) if not above.all() else None
        if k is None or k == 0:
            continue
        r0, r1 = ray[k - 1], ray[k]
        rs.append((k - 1) + (r0 - rm) / (r0 - r1))
    return float(np.mean(rs))


def laplace_pressure(rho, T, center=None):
    """Pressure jump P_EOS(rho at the centre) - P_EOS(rho at the far corner).
    The bulk pressure c_s^2 rho + G psi^2 equals P_EOS by Eq. (DED)."""
    ny, nx = rho.shape
    cx, cy = (nx // 2, ny // 2) if center is None else center
    return float(eos_pressure(rho[cy, cx], T) - eos_pressure(rho[0, 0], T))


def surface_tension_fit(radii, dps):
    """Least-squares slope and intercept of dP against 1/R (Eq. YLR, 2-D)."""
    inv = 1.0 / np.asarray(radii, dtype=float)
    A = np.vstack([inv, np.ones_like(inv)]).T
    (slope, icpt), *_ = np.linalg.lstsq(A, np.asarray(dps, dtype=float), rcond=None)
    return float(slope), float(icpt)
