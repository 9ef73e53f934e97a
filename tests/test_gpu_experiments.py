"""The paper's experiments of Sec. IV, run on the CUDA path through the C ABI.

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
