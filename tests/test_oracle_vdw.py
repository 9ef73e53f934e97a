"""Pins of the oracle's second equation of state, van der Waals.

Eq. (DED) turns any P_EOS(rho) into the pseudopotential psi; the paper uses
Carnahan-Starling (Eq. CSEOS), and the oracle also carries the van der Waals
equation in the same constants, P = k [c rho T / (1 - b rho) - a rho^2] with
a = 3, b = 1/3, c = 8/3: the reduced equation P/k = 8 rho T / (3 - rho) -
3 rho^2 of the textbooks.  The pins use what that equation fixes on its own:
values of the reduced equation worked by hand, its critical point (1, 1, k),
the mean-field shape of its coexistence curve next to the critical point,
and the mechanical-stability coexistence of the method (Eq. PGLDR) that a
flat interface of the oracle must relax to.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import theory


def test_vdw_pressure_is_the_reduced_equation():
    # 8 rho T/(3 - rho) - 3 rho^2, worked by hand, times k = 0.01
    cases = [(1.0, 1.0, 1.0),         # 8/2 - 3
             (1.5, 0.9, 0.45),        # 7.2 - 6.75
             (0.5, 0.8, 0.53),        # 1.28 - 0.75
             (2.0, 0.7, -0.8),        # 11.2 - 12
             (0.25, 0.6, 0.2488636363636364)]  # 1.2/2.75 - 0.1875
    for rho, T, want in cases:
        p = oracle.params(T=T, eos_kind="vdw")
        assert abs(oracle.eos_pressure(p, rho) - 0.01 * want) <= 1e-15, (rho, T)
        assert abs(theory.eos_pressure(rho, T, kind="vdw") - 0.01 * want) <= 1e-15, (rho, T)


def test_vdw_critical_point():
    rc, tc, pc = theory.critical_point(kind="vdw")
    assert abs(rc - 1.0) < 1e-8 and abs(tc - 1.0) < 1e-8 and abs(pc - 0.01) < 1e-12


def test_vdw_coexistence_next_to_the_critical_point():
    # mean field: rho_l - rho_g = 4 (1 - T)^(1/2) and the diameter
    # (rho_l + rho_g)/2 = 1 + 2/5 (1 - T) to leading order in 1 - T
    T = 0.999
    rg, rl = theory.maxwell(T, kind="vdw")
    assert abs((rl - rg) / (4.0 * math.sqrt(1.0 - T)) - 1.0) < 1e-3
    assert abs(((rl + rg) / 2.0 - 1.0) / (1.0 - T) - 0.4) < 1e-2
    # equal pressures at the two densities (the construction's condition)
    assert abs(theory.eos_pressure(rg, T, kind="vdw") - theory.eos_pressure(rl, T, kind="vdw")) < 1e-15


def test_vdw_psi_domain_and_value():
    # psi^2 = (P - rho/3)/G, positive through both phases at T_r 0.6..0.95
    for T in (0.6, 0.8, 0.95):
        rg, rl = theory.maxwell(T, kind="vdw")
        p = oracle.params(T=T, eos_kind="vdw")
        r = np.linspace(0.5 * rg, min(1.2 * rl, 2.9), 200)
        ps = oracle.psi(p, r)
        assert np.all(np.isfinite(ps)) and np.all(ps > 0)
        assert np.allclose(ps ** 2, -(np.array([oracle.eos_pressure(p, x) for x in r]) - r / 3.0),
                           rtol=1e-13, atol=0)


@pytest.mark.slow
def test_vdw_flat_interface_matches_pgldr():
    # a flat liquid band with the van der Waals EOS at T_r = 0.8, eps = 1.73,
    # relaxes to the coexistence that Eq. (PGLDR) predicts for that EOS
    from test_oracle_physics import _run_to_steady

    T = 0.8
    mg, ml = theory.maxwell(T, kind="vdw")
    rho = np.full((96, 2), mg)
    rho[24:72, :] = ml
    p = oracle.params(T=T, tau=1.0, eps=1.73, sigma=1.0, eos_kind="vdw")
    r, _, _ = _run_to_steady(p, rho, tol=1e-9)
    tg, tl = theory.pgldr(T, 1.73, kind="vdw")
    assert abs(r[48, 0] - tl) / tl < 5e-4
    assert abs(r[0, 0] - tg) / tg < 1.5e-2
