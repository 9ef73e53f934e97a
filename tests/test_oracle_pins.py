"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each check is a printed
number of the paper, a closed form, an exact identity of the scheme, an
independent brute-force evaluation, or a symmetry.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import theory
import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _rand_field(seed, ny, nx, lo, hi):
    return synth.uniform(seed, nx * ny, lo, hi).reshape(ny, nx)


# --------------------------------------------------------------------------- EOS / theory


def test_cs_critical_point_is_reduced_units():
    # With the printed a, b, c the Carnahan-Starling critical point sits at
    # rho_c = T_c = 1 and P_c = k: T in Eq. (CSEOS) is the reduced temperature.
    rc, tc, pc = theory.critical_point()
    assert abs(rc - 1.0) < 1e-6 and abs(tc - 1.0) < 1e-6 and abs(pc - 0.01) < 1e-8


def test_c_eos_matches_python_eos():
    # the C oracle's EOS and psi agree with the numpy theory module at many densities
    p = oracle.params(T=0.7)
    rho = np.linspace(0.01, 3.3, 101)
    c = np.array([oracle.eos_pressure(p, r) for r in rho])
    np.testing.assert_allclose(c, theory.eos_pressure(rho, 0.7), rtol=1e-12, atol=1e-16)
    np.testing.assert_allclose(oracle.psi(p, rho), theory.psi(rho, 0.7), rtol=1e-12)


def test_psi_domain_errors():
    p = oracle.params(T=0.8)
    bad = oracle.psi(p, np.array([-1.0, 0.0, 1.0 / oracle.CS_B, np.nan, np.inf]))
    assert np.isnan(bad).all()


def test_maxwell_matches_paper():
    g = GOLD["maxwell_Tr0.8"]
    rg, rl = theory.maxwell(0.8)
    assert round(rg, 4) == g["rho_g"] and round(rl, 4) == g["rho_l"]


def test_pgldr_matches_paper():
    g = GOLD["pgldr_Tr0.8_eps1.73"]
    rg, rl = theory.pgldr(0.8, 1.73)
    # printed with "approximately" to four decimals
    assert abs(rg - g["rho_g"]) <= 1e-4 and abs(rl - g["rho_l"]) <= 1e-4


def test_pgldr_eps_zero_is_not_maxwell():
    # plain Shan-Chen + Guo (eps = 0) is thermodynamically inconsistent: its
    # vapour density is far below Maxwell's (motivation of Sec. III).
    rg0, _ = theory.pgldr(0.8, 0.0)
    rgm, _ = theory.maxwell(0.8)
    assert rg0 < 0.5 * rgm


def test_lamb_period_matches_paper():
    g = GOLD["lamb_period"]
    pr = GOLD["table_prcases"]
    for t in ("0.6", "0.7"):
        ta = theory.lamb_period(pr[t]["gamma"], pr[t]["rho_l"], g["r_max"], g["r_min"])
        assert abs(ta - g[t]) < 0.5, (t, ta)


# --------------------------------------------------------------------------- force stencil


@pytest.mark.parametrize("eps", [0.0, 1.73])
@pytest.mark.parametrize("sigma", [0.125, 1.0, 4.0])
def test_force_moments_equal_bruteforce_aij(eps, sigma):
    # P3: the moment path (Eqs. FOMED, SOMED, DFTCCC, DFTCST, IFT) equals the
    # double sum over the A_ij tensor (Eq. Ansatz) on a 4x4 periodic lattice.
    p = oracle.params(T=0.8, eps=eps, sigma=sigma)
    rg, rl = theory.maxwell(0.8)
    rho = _rand_field(11, 4, 4, rg, rl)
    ps = oracle.psi(p, rho)
    fx, fy = oracle.force_moments(p, ps)
    bx, by = oracle.force_brute(p, ps)
    scale = max(np.abs(bx).max(), np.abs(by).max())
    assert np.abs(fx - bx).max() <= 1e-13 * scale
    assert np.abs(fy - by).max() <= 1e-13 * scale


def _quadratic(nx, ny, c):
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    a0, ax, ay, axx, axy, ayy = c
    psi = a0 + ax * x + ay * y + axx * x * x + axy * x * y + ayy * y * y
    gx = ax + 2 * axx * x + axy * y
    gy = ay + axy * x + 2 * ayy * y
    return psi, gx, gy, 2 * axx, axy, 2 * ayy


@pytest.mark.parametrize("variant", [0, 1])
def test_force_exact_on_quadratic_psi(variant):
    # P4: for a quadratic psi the D2Q9 moments are exact, M1 = c_s^2 grad psi,
    # M2 = c_s^4 grad grad psi, M0 - psi = c_s^2/2 lap psi, so Eq. (IFT)
    # equals its continuum form (Eqs. CFSCF leading term, CCFT, SSTFT):
    # F = -2 G psi grad psi - (3/4) eps c_s^2 G F1 + (sigma-1) c_s^2 G F2,
    # F1_a = -2 d_b psi d_a d_b psi,  F2_a = d_a psi lap psi - d_b psi d_a d_b psi.
    nx = ny = 9
    psi, gx, gy, hxx, hxy, hyy = _quadratic(nx, ny, (0.9, 0.013, -0.021, 0.0011, -0.0007, 0.0016))
    lap = hxx + hyy
    cs2 = 1 / 3
    for eps, sigma in [(0.0, 1.0), (1.73, 1.0), (1.73, 2.5), (0.4, 0.2)]:
        p = oracle.params(eps=eps, sigma=sigma, m2_trace_variant=variant)
        fx, fy = oracle.force_moments(p, psi)
        G = -1.0
        f1x = -2 * (gx * hxx + gy * hxy)
        f1y = -2 * (gx * hxy + gy * hyy)
        f2x = gx * lap - (gx * hxx + gy * hxy)
        f2y = gy * lap - (gx * hxy + gy * hyy)
        ex = -2 * G * psi * gx - 0.75 * eps * cs2 * G * f1x + (sigma - 1) * cs2 * G * f2x
        ey = -2 * G * psi * gy - 0.75 * eps * cs2 * G * f1y + (sigma - 1) * cs2 * G * f2y
        inner = (slice(1, ny - 1), slice(1, nx - 1))  # stencil does not wrap there
        np.testing.assert_allclose(fx[inner], ex[inner], rtol=0, atol=1e-14)
        np.testing.assert_allclose(fy[inner], ey[inner], rtol=0, atol=1e-14)


def test_alternative_trace_differs_on_general_field():
    # The two traces named after Eq. (DFTCST) agree on quadratics but are not
    # the same discrete operator: on a random field they differ.
    rho = _rand_field(5, 8, 8, 0.2, 2.3)
    p0 = oracle.params(sigma=2.0, m2_trace_variant=0)
    p1 = oracle.params(sigma=2.0, m2_trace_variant=1)
    ps = oracle.psi(p0, rho)
    a = oracle.force_moments(p0, ps)[0]
    b = oracle.force_moments(p1, ps)[0]
    assert np.abs(a - b).max() > 1e-6


@pytest.mark.parametrize("eps,sigma", [(0.0, 1.0), (1.73, 1.0), (0.0, 2.0), (1.73, 0.125)])
def test_total_force_vanishes_on_periodic_lattice(eps, sigma):
    # Every term of Eq. (IFT) carries an odd number of lattice velocities
    # (psi M1, M1 M2), while sum_x psi(x+c_i) psi(x+c_j) depends only on
    # c_j - c_i and is even in it; reversing all velocities therefore negates
    # the lattice sum of the force, which must vanish: momentum is conserved.
    rho = _rand_field(7, 16, 12, 0.2, 2.3)
    p = oracle.params(eps=eps, sigma=sigma)
    fx, fy = oracle.force_moments(p, oracle.psi(p, rho))
    s = np.abs(fx).sum() + np.abs(fy).sum()
    assert abs(fx.sum()) <= 1e-14 * s and abs(fy.sum()) <= 1e-14 * s


def test_shan_chen_special_case():
    # P5: eps = 0, sigma = 1 reduces Eq. (IFT) to Eq. (SCF) (Sec. IV.A); the
    # brute-force tensor then has only its j = 0 column: F = -(2G/c_s^2) psi
    # sum_i w_i c_i psi_i, checked here against a direct neighbour sum.
    rho = _rand_field(8, 6, 7, 0.2, 2.3)
    p = oracle.params(eps=0.0, sigma=1.0)
    ps = oracle.psi(p, rho)
    fx, fy = oracle.force_brute(p, ps)
    # Shan-Chen as the plain 8-neighbour difference stencil
    r = lambda dx, dy: np.roll(np.roll(ps, -dy, axis=0), -dx, axis=1)  # psi(x + (dx,dy))
    sx = (4 * (r(1, 0) - r(-1, 0)) + r(1, 1) - r(-1, 1) - r(-1, -1) + r(1, -1)) / 36.0
    sy = (4 * (r(0, 1) - r(0, -1)) + r(1, 1) + r(-1, 1) - r(-1, -1) - r(1, -1)) / 36.0
    np.testing.assert_allclose(fx, 6.0 * ps * sx, rtol=0, atol=1e-14)
    np.testing.assert_allclose(fy, 6.0 * ps * sy, rtol=0, atol=1e-14)


def test_force_d4_symmetry():
    # P6: transposing (x <-> y) and mirroring the psi field transposes /
    # mirrors the force, with the matching component sign changes.
    rho = _rand_field(9, 10, 10, 0.2, 2.3)
    p = oracle.params(eps=1.73, sigma=2.0)
    ps = oracle.psi(p, rho)
    fx, fy = oracle.force_moments(p, ps)
    tx, ty = oracle.force_moments(p, ps.T.copy())
    np.testing.assert_allclose(tx, fy.T, rtol=0, atol=1e-15)
    np.testing.assert_allclose(ty, fx.T, rtol=0, atol=1e-15)
    mir = np.roll(ps[:, ::-1], 1, axis=1)  # x -> -x (mod nx)
    mx, my = oracle.force_moments(p, mir)
    np.testing.assert_allclose(mx, -np.roll(fx[:, ::-1], 1, axis=1), rtol=0, atol=1e-15)
    np.testing.assert_allclose(my, np.roll(fy[:, ::-1], 1, axis=1), rtol=0, atol=1e-15)


# --------------------------------------------------------------------------- collision / step


def test_mrt_appendix_moment_vectors():
    # Appendix A prints M f^eq and M S for the Gram-Schmidt matrix; the
    # oracle's equilibrium (Eq. SEDF) and raw Guo term (Eq. GFS) must give them.
    M = np.array([[1, 1, 1, 1, 1, 1, 1, 1, 1], [-4, -1, -1, -1, -1, 2, 2, 2, 2],
                  [4, -2, -2, -2, -2, 1, 1, 1, 1], [0, 1, 0, -1, 0, 1, -1, -1, 1],
                  [0, -2, 0, 2, 0, 1, -1, -1, 1], [0, 0, 1, 0, -1, 1, 1, -1, -1],
                  [0, 0, -2, 0, 2, 1, 1, -1, -1], [0, 1, -1, 1, -1, 0, 0, 0, 0],
                  [0, 0, 0, 0, 0, 1, -1, 1, -1]], dtype=float)
    rho, ux, uy, Fx, Fy = 1.7, 0.031, -0.017, 0.0023, -0.0041
    feq, s = oracle.site_terms(rho, ux, uy, Fx, Fy)
    u2 = ux * ux + uy * uy
    meq = [rho, -2 * rho + 3 * rho * u2, rho - 3 * rho * u2, rho * ux, -rho * ux, rho * uy,
           -rho * uy, rho * (ux * ux - uy * uy), rho * ux * uy]
    uF = ux * Fx + uy * Fy
    sbar = [0, 6 * uF, -6 * uF, Fx, -Fx, Fy, -Fy, 2 * (ux * Fx - uy * Fy), ux * Fy + uy * Fx]
    np.testing.assert_allclose(M @ feq, meq, rtol=0, atol=1e-15)
    np.testing.assert_allclose(M @ s, sbar, rtol=0, atol=1e-15)


def test_mrt_with_equal_rates_is_bgk():
    # Sec. II.A: MRT recovers BGK when every relaxation rate equals 1/tau.
    rho = synth.droplet(24, 24, 7.0, 0.8)
    tau = 0.8
    a = oracle.run(oracle.params(tau=tau), rho, 30)
    b = oracle.run(oracle.params(tau=tau, collision="mrt", mrt_rates=[1 / tau] * 9), rho, 30)
    np.testing.assert_allclose(b["f"], a["f"], rtol=0, atol=1e-13)


def test_uniform_state_is_fixed_point():
    # P2: uniform rho, u = 0 => M1 = 0 => F = 0 and f = f^eq: nothing moves.
    rho = np.full((6, 5), 1.234)
    p = oracle.params(T=0.8)
    f0 = oracle.init_equilibrium(rho)
    f = oracle.step(p, f0.copy(), 50)
    # F and u are exactly zero; f only moves by the rounding of sum_i w_i rho
    assert (np.abs(f - f0) <= 2e-15 * f0).all()
    m = oracle.moments(p, f)
    assert np.abs(m["ux"]).max() == 0.0 and np.abs(m["Fx"]).max() == 0.0


def test_mass_conservation_exact():
    # P1: sum_i S_i = 0, sum_i (f_i - feq_i) = 0 and streaming permutes
    # values, so the total mass is conserved to rounding.
    rho = synth.droplet(32, 32, 9.0, 0.7)
    p = oracle.params(T=0.7, tau=1.0)
    f = oracle.init_equilibrium(rho)
    m0 = oracle.mass(f)
    oracle.step(p, f, 500)
    assert abs(oracle.mass(f) - m0) / m0 <= 1e-13


def test_step_d4_symmetry():
    # transposing the initial field transposes the state after many steps
    rho = synth.ellipse(20, 20, 7.0, 5.0, 0.8) + 0.01 * _rand_field(3, 20, 20, -1, 1)
    p = oracle.params(T=0.8, sigma=1.5)
    a = oracle.run(p, rho, 40)
    b = oracle.run(p, rho.T.copy(), 40)
    np.testing.assert_allclose(b["rho"], a["rho"].T, rtol=1e-13)
    np.testing.assert_allclose(b["ux"], a["uy"].T, rtol=0, atol=1e-14)


def test_oracle_reports_undefined_psi():
    rho = np.full((4, 4), 1.0)
    rho[1, 1] = 8.0  # b * rho > 1: outside the CS EOS domain
    with pytest.raises(oracle.OracleNumericError):
        oracle.run(oracle.params(), rho, 1)


def test_thread_count_does_not_change_results():
    rho = synth.droplet(24, 20, 6.0, 0.8)
    p = oracle.params(T=0.8)
    n0 = oracle.num_threads()
    try:
        oracle.set_num_threads(1)
        a = oracle.run(p, rho, 20)
        oracle.set_num_threads(max(2, n0))
        b = oracle.run(p, rho, 20)
    finally:
        oracle.set_num_threads(n0)
    assert np.array_equal(a["f"], b["f"]) and a["mass"] == b["mass"]
