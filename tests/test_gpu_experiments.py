"""The paper's experiments of Sec. IV, run on the CUDA path through the C ABI.

Fig. SDCC (Sec. IV.A) is the coexistence curve of a planar interface over
temperature, for plain Shan-Chen and the proposed force; its twelve flat
bands run as one batch handle and are compared with the FP64 oracle and
with Eq. (PGLDR).

Table DVT (the Young-Laplace test of Sec. IV.B) is a sweep over sigma. Its six
droplets are independent lattices, so they run as one batch handle: one
persistent launch per step over all six. Each lattice is read every 100
steps until Eq. (SSC) holds, as in the paper. Surface tension, gas and liquid
densities are then compared with the printed table.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import theory
import synth

pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table_dvt.json")))


@pytest.fixture(scope="module")
def P():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2003_07968_gb300 import build, capi

    build.build()
    capi.load()
    return capi


def test_table_dvt_sigma_sweep_in_one_batch(P):
    # Table DVT: droplet R0 = 50 on 200 x 200, BGK tau = 0.8, T_r = 0.8,
    # eps = 1.73, Maxwell initial densities; gamma = Delta P * R (Eq. YLR,
    # 2-D) with the interface at rho_m
    rows = GOLD["rows"]
    keys = list(rows)
    n = 200
    descs = [P.lbm_desc_default(n, n, T=0.8, tau=0.8, eps=1.73, sigma=float(Fraction(k)))
             for k in keys]
    h = P.lbm_create(descs)
    rho0 = synth.droplet(n, n, 50.0, 0.8)
    for i in range(len(keys)):
        P.lbm_init(h, i, rho0)
    prev = [None] * len(keys)
    steady = {}
    for k in range(600):
        P.lbm_step(h, 100)
        for i in range(len(keys)):
            if i in steady:
                continue
            r = P.lbm_moments(h, i, u=False, mass=False)["rho"]
            if prev[i] is not None and theory.steady_state_metric(r, prev[i]) < 1e-6:
                steady[i] = r
            prev[i] = r
        if len(steady) == len(keys):
            break
    P.lbm_destroy(h)
    assert len(steady) == len(keys), "no steady state within 60000 steps"
    for i, key in enumerate(keys):
        r, row = steady[i], rows[key]
        rg, rl = r[0, 0], r[n // 2, n // 2]
        R = theory.droplet_radius(r, rl, rg)
        gamma = theory.laplace_pressure(r, 0.8) * R
        # printed to four decimals.  For sigma = 4 the FP64 oracle, run the
        # same way, gives 0.05905: 99.7 % of gamma_pi (the paper prints 0.0603,
        # 101.9 %) with the printed densities to four decimals; that cell is
        # held to 2.5 %
        tol = 0.025 * row["gamma"] if key == "4" else 1.5e-4
        assert abs(gamma - row["gamma"]) <= tol, (key, gamma)
        assert abs(rg - row["rho_g"]) <= 1.5e-4, (key, rg)
        assert abs(rl - row["rho_l"]) <= 1.5e-4, (key, rl)


def test_coexistence_curve_fig_sdcc_in_one_batch(P):
    # Fig. SDCC: planar interfaces over temperature, plain Shan-Chen (eps = 0)
    # and the proposed force (eps = 1.73), BGK tau = 0.8.  Twelve flat bands in
    # one batch handle (32 x 128 each), 60000 steps, against the FP64 oracle
    # run the same way on 2 x 128 (a flat band is uniform in x, so the
    # discrete problem is the same).  Plain Shan-Chen started from the
    # Maxwell densities breaks down below T_r = 0.8 (in the oracle too), so
    # its curve starts there; where it runs, it sits on the mechanical-
    # stability densities of Eq. (PGLDR) with eps = 0.
    cases = [(0.0, T) for T in (0.8, 0.85, 0.9, 0.95)] + \
            [(1.73, T) for T in (0.6, 0.65, 0.7, 0.75, 0.8, 0.85, 0.9, 0.95)]
    steps = 60000
    descs = [P.lbm_desc_default(32, 128, T=T, tau=0.8, eps=eps, sigma=1.0) for eps, T in cases]
    h = P.lbm_create(descs)
    for i, (eps, T) in enumerate(cases):
        P.lbm_init(h, i, synth.band(32, 128, T, 32, 96))
    P.lbm_step(h, steps)
    got = [P.lbm_moments(h, i, u=False, mass=False)["rho"] for i in range(len(cases))]
    P.lbm_destroy(h)
    for (eps, T), g in zip(cases, got):
        o = oracle.run(oracle.params(T=T, tau=0.8, eps=eps, sigma=1.0),
                       synth.band(2, 128, T, 32, 96), steps)["rho"]
        gl, gg, ol, og = g[64, 0], g[0, 0], o[64, 0], o[0, 0]
        assert np.ptp(g, axis=1).max() <= 1e-6 * gl, (eps, T)  # still uniform in x
        assert abs(gl - ol) <= 1e-5 * ol, (eps, T, gl, ol)
        assert abs(gg - og) <= 1e-4 * og, (eps, T, gg, og)
        tg, tl = theory.pgldr(T, eps)
        if eps == 0.0:
            assert abs(ol - tl) <= 1e-4 * tl and abs(og - tg) <= 1e-3 * tg, (T, ol, og)
        else:
            # the liquid branch follows Eq. (PGLDR) closely at every T; the
            # vapour branch departs as the density ratio grows
            assert abs(ol - tl) <= 5e-4 * tl, (T, ol, tl)
            if T >= 0.8:
                assert abs(og - tg) <= 1e-2 * tg, (T, og, tg)


# Laplace law of configuration 2 against the planar surface tension.  The
# FP64 oracle, run the same way (tests/golden/make_config2_laplace.py), fits
# gamma at 0.969, 0.934, 0.933 and 0.891 of gamma_pi for T_r = 0.6, 0.7, 0.8,
# 0.9, with intercepts of 0.0, 1.3, 2.8 and 5.0 % of the largest Delta P:
# finite radii, and for T_r = 0.6 a largest droplet still relaxing after the
# 20000 steps.  The bounds sit just outside those.
GAMMA_TOL = {0.6: 0.05, 0.7: 0.10, 0.8: 0.10, 0.9: 0.15}
ICPT_TOL = 0.08
C2_PATH = os.path.join(os.path.dirname(__file__), "golden", "config2_laplace.json")


def test_config2_laplace_law_in_one_batch(P):
    # configuration 2: droplets R0 = 20 .. 60 on 256^2 at T_r = 0.6 .. 0.9, BGK
    # tau = 1, 20000 steps, all twenty in one batch handle.
    #  - each droplet against the oracle: whether it survived (R0 = 20 evaporates
    #    at T_r 0.8 and 0.9), and its densities, radius and Delta P within 1e-3;
    #  - per temperature, Delta P against 1/R over the surviving droplets
    #    (Eq. YLR in 2-D) is a line through about the origin whose slope, the
    #    surface tension, is compared with gamma_pi of the planar interface
    #    (Eqs. PTNNPI, STPI; the oracle's theory on a domain wide enough for
    #    the tails)
    C2 = json.load(open(C2_PATH))
    ref = C2["droplets"]
    n, steps = C2["n"], C2["steps"]
    h = P.lbm_create([P.lbm_desc_default(n, n, T=d["T"], tau=C2["tau"]) for d in ref])
    for i, d in enumerate(ref):
        P.lbm_init(h, i, synth.droplet(n, n, float(d["R0"]), d["T"]))
    P.lbm_step(h, steps)
    rho = [P.lbm_moments(h, i, u=False, mass=False)["rho"] for i in range(len(ref))]
    P.lbm_destroy(h)
    fits = {}
    for d, r in zip(ref, rho):
        rl, rg = r[n // 2, n // 2], r[0, 0]
        mg, ml = theory.maxwell(d["T"])
        assert (rl > 0.5 * (mg + ml)) == d["survived"], d
        assert abs(rl / d["rho_centre"] - 1) <= 1e-3 and abs(rg / d["rho_corner"] - 1) <= 1e-3, d
        if not d["survived"]:
            continue
        R, dP = theory.droplet_radius(r, rl, rg), theory.laplace_pressure(r, d["T"])
        assert abs(R / d["R"] - 1) <= 1e-3 and abs(dP / d["dP"] - 1) <= 1e-3, (d, R, dP)
        fits.setdefault(d["T"], []).append((R, dP))
    for T, pts in sorted(fits.items()):
        gamma, icpt = theory.surface_tension_fit([p[0] for p in pts], [p[1] for p in pts])
        gpi = theory.planar_interface(T, 1.73, 1.0, L=60.0, dx=0.05)[3]
        print(f"T_r {T}: {len(pts)} droplets, gamma {gamma:.5f} (planar {gpi:.5f}, "
              f"{gamma / gpi:.3f}), intercept {icpt:.2e}")
        assert abs(gamma / gpi - 1) <= GAMMA_TOL[T], (T, gamma, gpi)
        assert abs(icpt) <= ICPT_TOL * max(p[1] for p in pts), (T, icpt)
    # pin P8 as the survey states it: at T_r = 0.8 and R >= 40, the slope of
    # Delta P = gamma / R (Eq. YLR, a line through the origin) within 5 % of
    # the printed gamma_pi = 0.0148 (Sec. IV.B)
    big = [p for p in fits[0.8] if p[0] >= 38.0]
    x = np.array([1.0 / p[0] for p in big])
    y = np.array([p[1] for p in big])
    g8 = float(np.sum(x * y) / np.sum(x * x))
    print(f"T_r 0.8, R >= 40: gamma {g8:.5f} ({g8 / 0.0148:.3f} of 0.0148)")
    assert len(big) == 3 and abs(g8 / 0.0148 - 1) <= 0.05
