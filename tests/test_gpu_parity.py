"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: density within 1e-5 relative, pointwise (max_x |a-b|/|b|), for
FP32 population storage; FP16 deviation storage is held to its own, looser
stated bound.  Velocity is compared in absolute terms scaled by the largest
speed (|u| is tiny and sign-changing, so a pointwise relative norm is
meaningless there).
"""
import math
import time

import numpy as np
import pytest

import oracle
from oracle import theory
import synth

pytestmark = pytest.mark.gpu

RTOL_RHO = 1e-5


@pytest.fixture(scope="module")
def P():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2003_07968_gb300 import build, capi

    build.build()
    capi.load()
    return capi


def rel(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


def gpu_run(P, rho, nsteps, T=0.8, tau=1.0, eps=1.73, sigma=1.0, storage=None, eos=None,
            m2=0, tile=None, graph_steps=0, chunks=None, rho0=None, variant=0):
    ny, nx = rho.shape
    kw = dict(T=T, tau=tau, eps=eps, sigma=sigma, m2_trace_variant=m2)
    if storage is not None:
        kw["storage"] = storage
    if eos is not None:
        kw["eos_precision"] = eos
    if rho0 is not None:
        kw["rho0"] = rho0
    d = P.lbm_desc_default(nx, ny, **kw)
    h = P.lbm_create(d, tile=tile, graph_steps=graph_steps, kernel_variant=variant)
    P.lbm_init(h, 0, rho)
    for c in (chunks or [nsteps]):
        P.lbm_step(h, c)
    out = P.lbm_moments(h, 0)
    P.lbm_destroy(h)
    return out


def oracle_run(rho, nsteps, T=0.8, tau=1.0, eps=1.73, sigma=1.0, m2=0):
    return oracle.run(oracle.params(T=T, tau=tau, eps=eps, sigma=sigma, m2_trace_variant=m2),
                      rho, nsteps)


def test_config1_flat_band(P):
    # 64 x 64, liquid rows 16..47, T_r = 0.8, +-1e-3 noise, BGK tau = 1, 2000 steps
    rho = synth.flat_band(64, 64, 0.8)
    g1 = gpu_run(P, rho, 1000)
    o1 = oracle_run(rho, 1000)
    assert rel(g1["rho"], o1["rho"]) <= RTOL_RHO
    g2 = gpu_run(P, rho, 2000)
    o2 = oracle_run(rho, 2000)
    assert rel(g2["rho"], o2["rho"]) <= RTOL_RHO
    umax = np.abs(o2["ux"]).max() + np.abs(o2["uy"]).max()
    assert np.abs(g2["uy"] - o2["uy"]).max() <= 1e-3 * umax + 1e-9


@pytest.mark.parametrize("shape", [(2, 2), (4, 4), (7, 5), (3, 64), (37, 100), (33, 65)])
def test_small_and_ragged_lattices(P, shape):
    ny, nx = shape
    rg, rl = synth.coexistence(0.8)
    rho = synth.uniform(17 + nx * ny, nx * ny, rg, rl).reshape(ny, nx)
    # smooth the random field a little so the two-phase dynamics stay tame
    rho = 0.5 * rho + 0.5 * rho.mean()
    g = gpu_run(P, rho, 60)
    o = oracle_run(rho, 60)
    assert rel(g["rho"], o["rho"]) <= RTOL_RHO
    assert abs(g["mass"] - o["mass"]) / o["mass"] <= 1e-6


# kernel variants: 1 plain loads, 2 TMA pipeline
@pytest.mark.parametrize("variant,tile", [(2, (64, 8)), (2, (64, 16)), (2, (128, 4)),
                                          (2, (128, 8)), (2, (32, 16)), (1, (32, 1)),
                                          (1, (64, 2)), (1, (128, 4)), (1, (512, 1))])
def test_tile_shapes(P, variant, tile):
    rho = synth.droplet(97, 71, 20.0, 0.7)
    g = gpu_run(P, rho, 200, T=0.7, tile=tile, variant=variant)
    o = oracle_run(rho, 200, T=0.7)
    assert rel(g["rho"], o["rho"]) <= RTOL_RHO


def test_tma_and_plain_variants_agree(P):
    # same arithmetic, different summation order of rho in the psi pass:
    # they agree to the FP32 parity bar, not bitwise
    rho = synth.droplet(150, 130, 35.0, 0.7)
    a = gpu_run(P, rho, 300, T=0.7, variant=2)
    b = gpu_run(P, rho, 300, T=0.7, variant=1)
    assert rel(a["rho"], b["rho"]) <= RTOL_RHO


@pytest.mark.parametrize("eos", [0, 1, 2])
@pytest.mark.parametrize("storage", [0, 1])
def test_eos_precision_and_fp32_storage(P, eos, storage):
    rho = synth.droplet(80, 80, 22.0, 0.6)
    g = gpu_run(P, rho, 1000, T=0.6, eos=eos, storage=storage)
    o = oracle_run(rho, 1000, T=0.6)
    assert rel(g["rho"], o["rho"]) <= RTOL_RHO


@pytest.mark.parametrize("T", [0.8, 0.6])
def test_fp16_deviation_storage_stated_error(P, T):
    # FP16 keeps 11 significant bits, so this storage has its own stated
    # bound, not the FP32 one: after 1000 steps, 2e-3 relative in the bulk
    # phases and 1e-2 anywhere (automatic rho0 = vapour density; measured
    # 5.5-6.6e-4 and 1.7-3.2e-3).
    n = 80
    rho = synth.droplet(n, n, 22.0, T)
    g = gpu_run(P, rho, 1000, T=T, storage=2)
    o = oracle_run(rho, 1000, T=T)
    e = np.abs(g["rho"] - o["rho"]) / o["rho"]
    bulk = max(e[0, 0], e[n // 2, n // 2])
    print(f"fp16 T={T}: max rel rho error {e.max():.3e}, bulk {bulk:.3e}")
    assert bulk <= 2e-3 and e.max() <= 1e-2


@pytest.mark.parametrize("eps,sigma,m2", [(0.0, 1.0, 0), (1.73, 4.0, 0), (1.73, 0.125, 0),
                                          (1.73, 2.0, 1)])
def test_force_parameters_and_trace_variant(P, eps, sigma, m2):
    rho = synth.droplet(64, 64, 16.0, 0.8)
    g = gpu_run(P, rho, 500, eps=eps, sigma=sigma, m2=m2)
    o = oracle_run(rho, 500, eps=eps, sigma=sigma, m2=m2)
    assert rel(g["rho"], o["rho"]) <= RTOL_RHO


def test_uniform_fixed_point(P):
    rho = np.full((40, 48), 1.3)
    g = gpu_run(P, rho, 300)
    assert rel(g["rho"], rho) <= 1e-6
    assert np.abs(g["ux"]).max() <= 1e-7 and np.abs(g["uy"]).max() <= 1e-7


def test_non_finite_initial_density_is_refused(P):
    # every value is checked (one threaded pass for a million or more): a NaN
    # or an infinity anywhere, not only in the first or smallest value
    for nx, ny in [(48, 40), (1100, 1000)]:
        d = P.lbm_desc_default(nx, ny, T=0.8)
        h = P.lbm_create(d)
        base = synth.droplet(nx, ny, nx / 4.0, 0.8)
        for bad, at in [(np.nan, -1), (np.inf, nx * ny // 2 + 3), (-np.inf, 5), (np.nan, 0)]:
            rho = base.copy()
            rho.flat[at] = bad
            with pytest.raises(P.LbmError) as err:
                P.lbm_init(h, 0, rho)
            assert err.value.code == P.LBM_ERR_ARG
        P.lbm_init(h, 0, base)  # the handle stays usable
        P.lbm_step(h, 2)
        assert np.isfinite(P.lbm_moments(h, 0, u=False, mass=False)["rho"]).all()
        P.lbm_destroy(h)
    srv = P.lbm_server_create(P.lbm_server_opts_default(arena_bytes=1 << 26))
    rho = synth.droplet(64, 64, 16.0, 0.8)
    rho[63, 63] = np.nan
    with pytest.raises(P.LbmError) as err:
        P.lbm_submit(srv, P.lbm_desc_default(64, 64, T=0.8), rho, 10)
    assert err.value.code == P.LBM_ERR_ARG
    P.lbm_server_destroy(srv)


def test_copy_timeout_is_reported_and_the_handle_recovers(P):
    # failure detection without a GPU fault: one tile's staging copy is
    # skipped, so the consumers' bounded wait for it runs out (each wait of
    # that launch gives up after about 0.1 s), the CTA's warps leave together
    # and the producer drains its copies; the step reports LBM_ERR_TIMEOUT,
    # re-initialising the lattice clears it, and the handle goes on to match
    # the oracle
    n = 128
    rho = synth.droplet(n, n, 30.0, 0.8)
    h = P.lbm_create(P.lbm_desc_default(n, n, T=0.8), kernel_variant=P.LBM_KERNEL_TMA)
    info = P.lbm_info(h)
    assert info["collide_variant"] == P.LBM_KERNEL_TMA and info["tensor_map"] == 1
    P.lbm_init(h, 0, rho)
    P.lbm_step(h, 3)
    P.lbm_sync(h)
    P.lbm_inject_copy_timeout(h, info["n_tiles"] // 2)
    t0 = time.time()
    P.lbm_step(h, 2)
    with pytest.raises(P.LbmError) as err:
        P.lbm_sync(h)
    waited = time.time() - t0
    assert err.value.code == P.LBM_ERR_TIMEOUT and P.lbm_status_detail(h) == 0
    print(f"copy timeout reported after {waited:.1f} s")
    assert 0.05 < waited < 30
    P.lbm_init(h, 0, rho)
    P.lbm_step(h, 200)
    got = P.lbm_moments(h, 0, mass=False)["rho"]
    P.lbm_destroy(h)
    assert rel(got, oracle_run(rho, 200)["rho"]) <= RTOL_RHO


def test_mass_drift_fp32(P):
    rho = synth.droplet(128, 128, 30.0, 0.7)
    d = P.lbm_desc_default(128, 128, T=0.7)
    h = P.lbm_create(d)
    P.lbm_init(h, 0, rho)
    m0 = P.lbm_mass(h, 0)
    P.lbm_step(h, 2000)
    m1 = P.lbm_mass(h, 0)
    # the reduction against an exactly rounded sum of the per-site densities
    # (site sums as float-float pairs in both kernels, grouped differently)
    rho_sites = P.lbm_moments(h, 0, u=False, mass=False)["rho"]
    P.lbm_destroy(h)
    assert abs(m1 - math.fsum(rho_sites.ravel())) <= 1e-12 * m1
    exact = oracle.mass(oracle.init_equilibrium(rho))
    assert abs(m0 - exact) / exact <= 1e-6  # FP32 rounding of the initial populations
    drift = abs(m1 - m0) / m0
    print(f"FP32 mass drift over 2000 steps: {drift:.3e}")
    assert drift <= 1e-5


def test_graph_equals_direct_launches_and_is_deterministic(P):
    rho = synth.droplet(96, 96, 25.0, 0.8)
    a = gpu_run(P, rho, 100, graph_steps=-1)
    b = gpu_run(P, rho, 100, graph_steps=32)
    c = gpu_run(P, rho, 100, graph_steps=16, chunks=[33, 1, 66])
    assert np.array_equal(a["rho"], b["rho"]) and np.array_equal(a["rho"], c["rho"])
    assert np.array_equal(a["ux"], c["ux"])


def test_batch_lattices_equal_their_standalone_runs(P):
    rec = synth.batch_recipe(n=6, side=(40, 130))
    descs, fields = [], []
    for r in rec:
        descs.append(P.lbm_desc_default(r["nx"], r["ny"], T=r["T"]))
        fields.append(synth.droplet(r["nx"], r["ny"], r["R"], r["T"]))
    h = P.lbm_create(descs)
    for i, f in enumerate(fields):
        P.lbm_init(h, i, f)
    P.lbm_step(h, 150)
    for i, (r, f) in enumerate(zip(rec, fields)):
        got = P.lbm_moments(h, i)
        alone = gpu_run(P, f, 150, T=r["T"])
        assert np.array_equal(got["rho"], alone["rho"]), i
        if i < 2:
            o = oracle_run(f, 150, T=r["T"])
            assert rel(got["rho"], o["rho"]) <= RTOL_RHO
    P.lbm_destroy(h)


def test_autotune_keeps_state(P):
    rho = synth.droplet(200, 120, 30.0, 0.7)
    d = P.lbm_desc_default(200, 120, T=0.7)
    h = P.lbm_create(d)
    P.lbm_init(h, 0, rho)
    P.lbm_step(h, 50)
    info = P.lbm_autotune(h, 2)
    P.lbm_step(h, 50)
    got = P.lbm_moments(h, 0)
    P.lbm_destroy(h)
    ref = gpu_run(P, rho, 100, T=0.7)
    assert info["tile_x"] * info["tile_y"] <= 512
    assert rel(got["rho"], ref["rho"]) <= 1e-6


def test_numeric_fault_is_reported_not_trapped(P):
    rho = np.full((16, 16), 1.0)
    rho[3, 5] = 8.5  # b * rho > 1: outside the Carnahan-Starling domain
    d = P.lbm_desc_default(16, 16)
    h = P.lbm_create(d)
    P.lbm_init(h, 0, rho)
    P.lbm_step(h, 1)
    with pytest.raises(P.LbmError) as ei:
        P.lbm_sync(h)
    assert ei.value.code == P.LBM_ERR_NUMERIC
    assert P.lbm_status_detail(h) == 0
    # re-initialising the lattice clears the fault
    P.lbm_init(h, 0, np.full((16, 16), 1.0))
    P.lbm_step(h, 3)
    P.lbm_sync(h)
    P.lbm_destroy(h)


def test_bad_arguments_are_rejected(P):
    with pytest.raises(P.LbmError):
        P.lbm_create(P.lbm_desc_default(1, 8))
    with pytest.raises(P.LbmError):
        P.lbm_create(P.lbm_desc_default(8, 8, tau=0.5))
    with pytest.raises(P.LbmError):
        P.lbm_create([P.lbm_desc_default(8, 8), P.lbm_desc_default(8, 8, storage=2)])
    h = P.lbm_create(P.lbm_desc_default(8, 8))
    with pytest.raises(P.LbmError):
        P.lbm_step(h, -1)
    P.lbm_destroy(h)


# ------------------------------------------------------------- full-size sampled parity
def _windows_oracle(rho_full, sites, nsteps, **kw):
    """Oracle value of rho at each sampled site after nsteps, computed on a
    window of half-width 2 nsteps + 2 around it: information moves at most
    two sites per step (one for the psi stencil, one for streaming), so what
    happens at the window's border cannot reach the centre.  The window is
    mirrored into a periodic field (no jump at its seams) so the oracle's
    periodic run stays inside the EOS domain there."""
    half = 2 * nsteps + 2
    out = []
    for (y, x) in sites:
        ys = np.arange(y - half, y + half + 1)
        xs = np.arange(x - half, x + half + 1)
        win = rho_full.take(ys, axis=0, mode="wrap").take(xs, axis=1, mode="wrap")
        per = np.concatenate([win, win[::-1]], axis=0)
        per = np.concatenate([per, per[:, ::-1]], axis=1)
        m = oracle_run(per, nsteps, **kw)
        out.append(m["rho"][half, half])
    return np.array(out)


def _sample_sites(nx, ny, n, seed):
    ys = synth.randint(seed, n, 0, ny - 1)
    xs = synth.randint(seed, n, 0, nx - 1, offset=n)
    edge = [(0, 0), (ny - 1, nx - 1), (0, nx - 1), (ny - 1, 0), (ny // 2, nx // 2)]
    return edge + list(zip(ys.tolist(), xs.tolist()))


@pytest.mark.parametrize("case", ["roofline_8192", "oscillating_1024"])
def test_full_size_sampled_parity(P, case):
    if case == "roofline_8192":
        n, T, tau = 8192, 0.8, 1.0
        rho = synth.droplet(n, n, 2048.0, T)
        tile = None
    else:
        n, T, tau = 1024, 0.6, 0.8
        rho = synth.ellipse(n, n, 120.0, 100.0, T)
        tile = None
    nsteps = 5
    g = gpu_run(P, rho, nsteps, T=T, tau=tau, tile=tile)
    sites = _sample_sites(n, n, 40, 99)
    # sample the interface too: rows crossing the droplet edge
    if case == "roofline_8192":
        sites += [(n // 2, n // 2 + 2048 + k) for k in range(-3, 4)]
    else:
        sites += [(n // 2, n // 2 + 120 + k) for k in range(-3, 4)]
    want = _windows_oracle(rho, sites, nsteps, T=T, tau=tau)
    got = np.array([g["rho"][y, x] for (y, x) in sites])
    assert rel(got, want) <= RTOL_RHO
    # a property that holds at any size: the total mass is conserved
    # (f = f^eq(rho, 0) at start, so the initial mass is sum_x rho)
    exact = float(rho.sum())
    assert abs(g["mass"] - exact) / exact <= 1e-6


def test_roofline_droplet_1000_steps_against_oracle_golden(P):
    # the 8192^2 droplet the throughput is measured on (R = 2048, T_r = 0.8,
    # tau = 1), 1000 steps in the launch configuration bench.py times
    # (autotuned single pass), against the FP64 oracle's values at 614
    # sampled sites (interface crossings along both axes and a diagonal,
    # corners, edges, centre, 200 seeded sites) and its total mass, written
    # by tests/golden/make_roofline_1000.py
    import json
    import os

    with open(os.path.join(os.path.dirname(__file__), "golden", "roofline_1000.json")) as fh:
        gold = json.load(fh)
    n, T, tau = gold["n"], gold["T"], gold["tau"]
    rho = synth.droplet(n, n, gold["R"], T)
    d = P.lbm_desc_default(n, n, T=T, tau=tau)
    h = P.lbm_create(d)
    P.lbm_init(h, 0, rho)
    P.lbm_autotune(h)  # trial launches leave the state unchanged
    P.lbm_step(h, gold["steps"])
    out = P.lbm_moments(h, 0, u=False)
    P.lbm_destroy(h)
    ys, xs, want = (np.array(c) for c in zip(*gold["sites"]))
    got = out["rho"][ys.astype(int), xs.astype(int)]
    err = rel(got, want)
    print(f"8192^2 droplet, 1000 steps, {len(want)} sampled sites: {err:.2e}")
    assert err <= RTOL_RHO
    assert abs(out["mass"] - gold["mass"]) / gold["mass"] <= 1e-9


# ------------------------------------------------------------- derived quantities
def test_config2_laplace_quantities(P):
    # 256 x 256 droplet R = 30 at T_r = 0.7, tau = 1, 20000 steps: coexistence
    # densities and the Laplace pressure jump within 1e-3 of the oracle.
    n, T, R = 256, 0.7, 30.0
    rho = synth.droplet(n, n, R, T)
    g = gpu_run(P, rho, 20000, T=T)["rho"]
    o = oracle_run(rho, 20000, T=T)["rho"]
    for name, a, b in [("rho_l", g[n // 2, n // 2], o[n // 2, n // 2]),
                       ("rho_g", g[0, 0], o[0, 0]),
                       ("dP", theory.laplace_pressure(g, T), theory.laplace_pressure(o, T))]:
        assert abs(a - b) / abs(b) <= 1e-3, name
    ra = theory.droplet_radius(g, g[n // 2, n // 2], g[0, 0])
    rb = theory.droplet_radius(o, o[n // 2, n // 2], o[0, 0])
    assert abs(ra - rb) / rb <= 1e-3


def _first_period(ext, every):
    """Period from the +x extremity sampled every `every` steps: the first
    minimum, then the next maximum (one full period after t = 0), located
    by a parabola through the seven samples around it."""
    ext = np.asarray(ext, dtype=float)
    t = every * np.arange(len(ext), dtype=float)
    k1 = int(np.argmin(ext[: len(ext) // 2 + 10]))
    k2 = k1 + int(np.argmax(ext[k1:]))
    a, b, _ = np.polyfit(t[k2 - 3:k2 + 4], ext[k2 - 3:k2 + 4], 2)
    return -b / (2 * a)


def test_config3_oscillation_period(P):
    # 1024 x 1024 ellipse 120/100 at T_r = 0.6, BGK tau = 0.8, 50000 steps,
    # the +x extremity sampled every 500 steps (Sec. IV.C): the period within
    # 1e-3 of the FP64 oracle's (tests/golden/config3_period.json, written by
    # make_config3_period.py), the sampled extremities within 0.02 sites of
    # the oracle's, and the period within 10 % of Lamb's Eq. (DOP) with the
    # paper's Table PRCases gamma and rho_l (BGK damping and the finite
    # interface width are not part of Lamb's result)
    import json
    import os

    with open(os.path.join(os.path.dirname(__file__), "golden", "config3_period.json")) as fh:
        gold = json.load(fh)
    n, T, every = gold["n"], gold["T"], gold["every"]
    rho = synth.ellipse(n, n, 120.0, 100.0, T)
    rg, rl = synth.coexistence(T)
    d = P.lbm_desc_default(n, n, T=T, tau=gold["tau"])
    h = P.lbm_create(d)
    P.lbm_init(h, 0, rho)
    ext = []
    rm = 0.5 * (rl + rg)
    for k in range(len(gold["extremity"])):
        if k:
            P.lbm_step(h, every)
        r = P.lbm_moments(h, 0, u=False, mass=False)["rho"]
        ray = r[n // 2, n // 2:]
        j = int(np.argmax(ray < rm))
        ext.append((j - 1) + (ray[j - 1] - rm) / (ray[j - 1] - ray[j]))
    P.lbm_destroy(h)
    period = _first_period(ext, every)
    want = _first_period(gold["extremity"], every)
    ta = theory.lamb_period(0.0461, 3.1192, 120.0, 100.0)
    dev = float(np.max(np.abs(np.array(ext) - np.array(gold["extremity"]))))
    print(f"oscillation period {period:.1f} steps (oracle {want:.1f}, Lamb {ta:.0f}); "
          f"extremities within {dev:.2e} sites of the oracle's")
    assert abs(period - want) / want <= 1e-3
    assert dev <= 0.02
    assert abs(period - ta) / ta <= 0.10


def test_config4_batch_of_512_against_oracle(P):
    # the 512-lattice uneven batch, 1000 steps in one handle; the smallest and
    # largest lattice and 16 seeded others against the oracle, every one held
    # to the FP32 bar
    rec = synth.batch_recipe()
    descs = [P.lbm_desc_default(r["nx"], r["ny"], T=r["T"]) for r in rec]
    fields = [synth.droplet(r["nx"], r["ny"], r["R"], r["T"]) for r in rec]
    h = P.lbm_create(descs)
    for i, f in enumerate(fields):
        P.lbm_init(h, i, f)
    P.lbm_step(h, 1000)
    sides = np.array([r["nx"] for r in rec])
    picks = [int(np.argmin(sides)), int(np.argmax(sides))] + synth.randint(77, 16, 0, 511).tolist()
    worst = 0.0
    for i in picks:
        got = P.lbm_moments(h, i, u=False, mass=False)["rho"]
        o = oracle_run(fields[i], 1000, T=rec[i]["T"])["rho"]
        err = rel(got, o)
        worst = max(worst, err)
        print(f"lattice {i} side {rec[i]['nx']} T {rec[i]['T']:.3f}: {err:.2e}")
        assert err <= RTOL_RHO, (i, rec[i], err)
    P.lbm_destroy(h)
    print(f"config 4: worst density error after 1000 steps {worst:.2e}")


def test_largest_batch_lattice_alone_both_fp32_storages(P):
    # the batch's 512^2 lattice (R = 170, T_r = 0.70) alone, with FP32
    # storage of deviations from rho0 = 0 and from the automatic rho0
    i = int(np.argmax([r["nx"] for r in synth.batch_recipe()]))
    r = synth.batch_recipe()[i]
    rho = synth.droplet(r["nx"], r["ny"], r["R"], r["T"])
    o = oracle_run(rho, 1000, T=r["T"])["rho"]
    for storage in (0, 1):
        g = gpu_run(P, rho, 1000, T=r["T"], storage=storage)["rho"]
        print(f"512^2 alone, storage {storage}: {rel(g, o):.2e}")
        assert rel(g, o) <= RTOL_RHO, storage


def test_config3_ellipse_1000_steps_full_field(P):
    # configuration 3 (1024^2 ellipse 120/100, T_r = 0.6, BGK tau = 0.8):
    # the whole density field after 1000 steps against the oracle at the FP32
    # bar, and both velocity components scaled by the largest speed
    n, T, tau = 1024, 0.6, 0.8
    rho = synth.ellipse(n, n, 120.0, 100.0, T)
    g = gpu_run(P, rho, 1000, T=T, tau=tau)
    o = oracle_run(rho, 1000, T=T, tau=tau)
    err = rel(g["rho"], o["rho"])
    print(f"1024^2 ellipse, 1000 steps: density {err:.2e}")
    assert err <= RTOL_RHO
    umax = max(np.abs(o["ux"]).max(), np.abs(o["uy"]).max())
    for k in ("ux", "uy"):
        assert np.abs(g[k] - o[k]).max() <= 1e-3 * umax, k
    assert abs(g["mass"] - o["mass"]) / o["mass"] <= 1e-9


@pytest.mark.parametrize("eos", [1, 0])
def test_fused_schedule(P, eos):
    # one pass per step, psi rebuilt on each tile's halo: bitwise the same
    # numbers as the two-pass step (every psi is the same sequence of rounded
    # operations on the same loaded values), and the oracle
    rho = synth.droplet(150, 110, 32.0, 0.7)
    outs = []
    for sched in (P.LBM_SCHED_TWO_PASS, P.LBM_SCHED_FUSED):
        d = P.lbm_desc_default(150, 110, T=0.7, eos_precision=eos)
        h = P.lbm_create(d, schedule=sched)
        P.lbm_init(h, 0, rho)
        P.lbm_step(h, 400)
        outs.append(P.lbm_moments(h, 0))
        P.lbm_destroy(h)
    assert np.array_equal(outs[1]["rho"], outs[0]["rho"])
    assert np.array_equal(outs[1]["ux"], outs[0]["ux"])
    o = oracle_run(rho, 400, T=0.7)
    assert rel(outs[1]["rho"], o["rho"]) <= RTOL_RHO


@pytest.mark.parametrize("eos", [0, 1, 2])
def test_sites_per_thread_are_bitwise_invariant(P, eos):
    # one site per thread (scalar FP32) and two or four (site pairs on the
    # paired FP32 instructions) run the same rounded operations per site
    rho = synth.droplet(131, 97, 30.0, 0.6)
    outs = []
    for sched, tile, spt in ((P.LBM_SCHED_FUSED, (32, 8), 1), (P.LBM_SCHED_FUSED, (32, 8), 2),
                             (P.LBM_SCHED_FUSED, (64, 8), 4), (P.LBM_SCHED_TWO_PASS, (64, 4), 2)):
        d = P.lbm_desc_default(131, 97, T=0.6, eos_precision=eos)
        h = P.lbm_create(d, schedule=sched, tile=tile, sites_per_thread=spt)
        assert P.lbm_info(h)["spt"] == spt
        P.lbm_init(h, 0, rho)
        P.lbm_step(h, 300)
        outs.append(P.lbm_moments(h, 0, mass=False))
        P.lbm_destroy(h)
    for o in outs[1:]:
        assert np.array_equal(o["rho"], outs[0]["rho"])
        assert np.array_equal(o["ux"], outs[0]["ux"])


def test_fused_batch_and_fault(P):
    rec = synth.batch_recipe(n=5, side=(30, 90))
    descs = [P.lbm_desc_default(r["nx"], r["ny"], T=r["T"]) for r in rec]
    fields = [synth.droplet(r["nx"], r["ny"], r["R"], r["T"]) for r in rec]
    h = P.lbm_create(descs, schedule=P.LBM_SCHED_FUSED)
    for i, f in enumerate(fields):
        P.lbm_init(h, i, f)
    P.lbm_step(h, 120)
    for i in (0, 4):
        o = oracle_run(fields[i], 120, T=rec[i]["T"])
        assert rel(P.lbm_moments(h, i)["rho"], o["rho"]) <= RTOL_RHO
    bad = fields[2].copy()
    bad[3, 3] = 8.5
    P.lbm_init(h, 2, bad)
    P.lbm_step(h, 1)
    with pytest.raises(P.LbmError) as ei:
        P.lbm_sync(h)
    assert ei.value.code == P.LBM_ERR_NUMERIC and P.lbm_status_detail(h) == 2
    P.lbm_destroy(h)


# ------------------------------------------------------------- MRT (Appendix A)
def mrt_desc(P, n, T, tau=0.65, rates=None):
    r = rates if rates is not None else [1.0] * 7 + [1.0 / tau] * 2
    return P.lbm_desc_default(n, n, T=T, tau=tau, collision=P.LBM_COLL_MRT, mrt_rates=r)


@pytest.mark.parametrize("sched", [0, 1])
def test_mrt_matches_oracle(P, sched):
    # the paper's dynamic test setup (Sec. IV.C): 200^2 ellipse 30/27, T_r=0.6,
    # MRT with Lambda = diag(1,...,1,1/tau,1/tau), tau = 0.65
    n, T = 200, 0.6
    rho = synth.ellipse(n, n, 30.0, 27.0, T)
    h = P.lbm_create(mrt_desc(P, n, T), schedule=sched)
    P.lbm_init(h, 0, rho)
    P.lbm_step(h, 1000)
    got = P.lbm_moments(h, 0)
    P.lbm_destroy(h)
    o = oracle.run(oracle.params(T=T, tau=0.65, collision="mrt"), rho, 1000)
    assert rel(got["rho"], o["rho"]) <= RTOL_RHO


def test_mrt_with_equal_rates_is_bgk(P):
    n, T, tau = 96, 0.7, 0.8
    rho = synth.droplet(n, n, 24.0, T)
    h = P.lbm_create(mrt_desc(P, n, T, tau=tau, rates=[1 / tau] * 9))
    P.lbm_init(h, 0, rho)
    P.lbm_step(h, 300)
    a = P.lbm_moments(h, 0)
    P.lbm_destroy(h)
    b = gpu_run(P, rho, 300, T=T, tau=tau)
    # two different FP32 evaluations of the same update (moment space vs the
    # paired-direction BGK form): measured 1.9e-6 apart after 300 steps, each
    # within 2.3e-6 of the FP64 oracle; held to the density bar
    assert rel(a["rho"], b["rho"]) <= RTOL_RHO


def test_mrt_oscillation_period_on_gpu(P):
    # Sec. IV.C: period 3200 at T_r = 0.6 (sampled every 100 steps there)
    n, T = 200, 0.6
    rg, rl = synth.coexistence(T)
    h = P.lbm_create(mrt_desc(P, n, T))
    P.lbm_init(h, 0, synth.ellipse(n, n, 30.0, 27.0, T))
    d = []
    for k in range(401):
        if k:
            P.lbm_step(h, 10)
        r = P.lbm_moments(h, 0, u=False, mass=False)["rho"]
        ray = r[n // 2, n // 2:]
        rm = 0.5 * (rl + rg)
        j = int(np.argmax(ray < rm))
        d.append((j - 1) + (ray[j - 1] - rm) / (ray[j - 1] - ray[j]))
    P.lbm_destroy(h)
    t = np.arange(401) * 10.0
    sm = np.convolve(np.array(d), np.ones(21) / 21, mode="same")
    win = (t >= 2000) & (t <= 3900)
    k = int(np.argmax(np.where(win, sm, -np.inf)))
    a, b, _ = np.polyfit(t[k - 15:k + 16], sm[k - 15:k + 16], 2)
    period = -b / (2 * a)
    print(f"MRT oscillation period on the GPU: {period:.0f} steps (paper: 3200)")
    assert abs(period - 3200) <= 100


@pytest.mark.parametrize("tile", [(64, 8), (32, 16), (64, 16), (128, 8)])
def test_fused_tma_equals_plain_fused_bitwise(P, tile):
    # the TMA-staged single pass runs the same per-site arithmetic on the same
    # values as the plain-load single pass: bitwise equal results, on ragged
    # lattices of a batch (tiles crossing the right and bottom edges)
    rec = synth.batch_recipe(n=4, side=(37, 150))
    descs = [P.lbm_desc_default(r["nx"], r["ny"], T=r["T"]) for r in rec]
    fields = [synth.droplet(r["nx"], r["ny"], r["R"], r["T"]) for r in rec]
    # a batch of similar widths shares one row space (one tensor map); a
    # lopsided batch keeps the compact layout (bulk row copies)
    lop = [(600, 40), (40, 600), (64, 64)]
    cases = [(descs, fields, 1),
             ([P.lbm_desc_default(nx, ny, T=0.7) for nx, ny in lop],
              [synth.droplet(nx, ny, min(nx, ny) / 3.0, 0.7) for nx, ny in lop], 0)]
    for dd, ff, tensor in cases:
        outs = []
        for variant, sp in ((P.LBM_KERNEL_PLAIN, 2), (P.LBM_KERNEL_TMA, 0)):
            h = P.lbm_create(dd, schedule=P.LBM_SCHED_FUSED, kernel_variant=variant, tile=tile,
                             sites_per_thread=sp if variant == P.LBM_KERNEL_PLAIN else 0)
            info = P.lbm_info(h)
            assert info["collide_variant"] == variant
            if variant == P.LBM_KERNEL_TMA:
                assert info["tensor_map"] == tensor
            for i, f in enumerate(ff):
                P.lbm_init(h, i, f)
            P.lbm_step(h, 150)
            outs.append([P.lbm_moments(h, i, mass=False) for i in range(len(dd))])
            P.lbm_destroy(h)
        for a, b in zip(*outs):
            assert np.array_equal(a["rho"], b["rho"]) and np.array_equal(a["ux"], b["ux"])
    o = oracle_run(fields[0], 150, T=rec[0]["T"])
    h = P.lbm_create(descs, schedule=P.LBM_SCHED_FUSED, kernel_variant=P.LBM_KERNEL_TMA, tile=tile)
    for i, f in enumerate(fields):
        P.lbm_init(h, i, f)
    P.lbm_step(h, 150)
    assert rel(P.lbm_moments(h, 0, mass=False)["rho"], o["rho"]) <= RTOL_RHO
    P.lbm_destroy(h)
    # a single ragged lattice takes the tensor-map path (one 3-D copy per tile)
    nx, ny = 203, 77
    rho = synth.droplet(nx, ny, 25.0, 0.7)
    single = []
    for variant, sp in ((P.LBM_KERNEL_PLAIN, 2), (P.LBM_KERNEL_TMA, 0)):
        h = P.lbm_create(P.lbm_desc_default(nx, ny, T=0.7), schedule=P.LBM_SCHED_FUSED,
                         kernel_variant=variant, tile=tile,
                         sites_per_thread=sp if variant == P.LBM_KERNEL_PLAIN else 0)
        if variant == P.LBM_KERNEL_TMA:
            assert P.lbm_info(h)["tensor_map"] == 1
        P.lbm_init(h, 0, rho)
        P.lbm_step(h, 150)
        single.append(P.lbm_moments(h, 0, mass=False))
        P.lbm_destroy(h)
    assert np.array_equal(single[0]["rho"], single[1]["rho"])
    assert np.array_equal(single[0]["ux"], single[1]["ux"])


@pytest.mark.parametrize("storage,mrt", [(2, False), (1, True)])
def test_fused_tma_storage_and_mrt(P, storage, mrt):
    n, T = 100, 0.7
    rho = synth.droplet(n, n, 24.0, T)
    kw = dict(T=T, storage=storage)
    if mrt:
        kw.update(collision=P.LBM_COLL_MRT, tau=0.8, mrt_rates=[1.0] * 7 + [1 / 0.8] * 2)
    outs = []
    for variant in (P.LBM_KERNEL_PLAIN, P.LBM_KERNEL_TMA):
        h = P.lbm_create(P.lbm_desc_default(n, n, **kw), schedule=P.LBM_SCHED_FUSED,
                         kernel_variant=variant, tile=(64, 8),
                         sites_per_thread=2 if variant == P.LBM_KERNEL_PLAIN else 0)
        P.lbm_init(h, 0, rho)
        P.lbm_step(h, 200)
        outs.append(P.lbm_moments(h, 0, mass=False))
        P.lbm_destroy(h)
    assert np.array_equal(outs[0]["rho"], outs[1]["rho"])


def test_step_reciprocal_and_square_root_error_bounds(P):
    # the kernels' 1/x and sqrt(x) (hardware approximation + one Newton step,
    # paired lanes) against correctly rounded float32 results over the ranges
    # the step uses them on: 1/rho and 1/(1 - b rho) (rho in (0, 8)), psi^2
    # (0 .. 30), plus tiny, huge, zero and power-of-two arguments
    rng = np.random.default_rng(2003)
    x = np.concatenate([
        rng.uniform(1e-3, 8.0, 200000), rng.uniform(0.05, 1.0, 200000),
        np.exp(rng.uniform(np.log(1e-37), np.log(1e37), 200000)),
        2.0 ** np.arange(-120, 121, dtype=np.float64), [1.0, 4.0, 0.25, 3.0, 7.0],
    ]).astype(np.float32)
    r, q = P.lbm_selfcheck_arith(x)  # raises LBM_ERR_STATE if paired != scalar lane

    def ulps(a, b):  # distance in units of the last place, same sign, finite
        ia = a.view(np.int32).astype(np.int64)
        ib = b.view(np.int32).astype(np.int64)
        return np.abs(ia - ib)

    normal = (x > 1.2e-38) & (x < 8.5e37)  # 1/x normal too
    exact_r = (np.float32(1.0) / x[normal]).astype(np.float32)
    exact_q = np.sqrt(x).astype(np.float32)
    er, eq = ulps(r[normal], exact_r), ulps(q, exact_q)
    print(f"1/x: max {er.max()} ulp, {np.mean(er == 0):.4f} exact; "
          f"sqrt: max {eq.max()} ulp, {np.mean(eq == 0):.4f} exact")
    assert er.max() <= 1 and eq.max() <= 1
    assert np.mean(er == 0) > 0.9 and np.mean(eq == 0) > 0.9
    # zero and the powers of two are exact
    r0, q0 = P.lbm_selfcheck_arith(np.array([0.0, 2.0 ** -130, 2.0 ** -140], np.float32))
    assert q0[0] == 0.0
    assert q0[1] == np.sqrt(np.float32(2.0 ** -130)) and q0[2] == np.float32(2.0 ** -70)
