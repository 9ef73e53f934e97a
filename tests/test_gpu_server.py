"""GPU tests of the continuous-batching server (lbm_submit / lbm_poll).

A result must not depend on what else was resident: every served lattice is
compared bitwise with the same lattice stepped alone by a handle that uses
the same kernels and tiles.
"""
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TILE = (32, 8)


@pytest.fixture(scope="module")
def P():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2003_07968_gb300 import build, capi

    build.build()
    capi.load()
    return capi


def alone(P, desc, rho, nsteps):
    h = P.lbm_create(desc, tile=TILE, kernel_variant=P.LBM_KERNEL_PLAIN)
    P.lbm_init(h, 0, rho)
    P.lbm_step(h, nsteps)
    out = P.lbm_moments(h, 0, mass=False)
    P.lbm_destroy(h)
    return out


def wait(P, srv, tickets, timeout=120.0):
    res = {}
    t0 = time.time()
    while len(res) < len(tickets):
        for t in tickets:
            if t not in res:
                r = P.lbm_poll(srv, t)
                if r is not None:
                    res[t] = r
        assert time.time() - t0 < timeout, "server did not finish"
        time.sleep(0.002)
    return res


def test_served_results_equal_alone_runs(P):
    # fixed chunks of 37 steps (chunk_ms < 0); the other tests run chunks
    # sized by GPU time, of varying length
    opts = P.lbm_server_opts_default(arena_bytes=1 << 30, chunk_steps=37, chunk_ms=-1.0,
                                     kernel_variant=P.LBM_KERNEL_PLAIN, tile_x=TILE[0],
                                     tile_y=TILE[1])
    srv = P.lbm_server_create(opts)
    specs = [(48, 40, 12.0, 0.8, 120), (130, 97, 30.0, 0.7, 260), (64, 64, 18.0, 0.6, 75),
             (200, 150, 40.0, 0.75, 300), (33, 65, 9.0, 0.85, 50), (96, 96, 24.0, 0.65, 190)]
    tickets, jobs = [], []
    for k, (nx, ny, R, T, n) in enumerate(specs):
        d = P.lbm_desc_default(nx, ny, T=T)
        rho = synth.droplet(nx, ny, R, T)
        tickets.append(P.lbm_submit(srv, d, rho, n))
        jobs.append((d, rho, n))
        if k == 2:
            time.sleep(0.05)  # later requests join while the first ones run
    res = wait(P, srv, tickets)
    st = P.lbm_server_get_stats(srv)
    assert st["completed"] == len(specs) and st["failed"] == 0
    assert st["site_steps"] == sum(nx * ny * n for nx, ny, _, _, n in specs)
    for t, (d, rho, n) in zip(tickets, jobs):
        a = alone(P, d, rho, n)
        assert np.array_equal(res[t]["rho"], a["rho"]), (d.nx, d.ny)
        assert np.array_equal(res[t]["ux"], a["ux"])
        assert res[t]["latency_s"] > 0
    # and one of them against the oracle
    d, rho, n = jobs[1]
    o = oracle.run(oracle.params(T=d.T), rho, n)
    assert np.max(np.abs(res[tickets[1]]["rho"] - o["rho"]) / o["rho"]) <= 1e-5
    P.lbm_server_destroy(srv)


def test_server_admission_capacity_and_failures(P):
    # a small arena: requests wait for space, one never fits, one fails alone
    opts = P.lbm_server_opts_default(arena_bytes=8 << 20, chunk_steps=20, max_resident=3,
                                     max_width=128)
    srv = P.lbm_server_create(opts)
    with pytest.raises(P.LbmError) as ei:
        big = P.lbm_desc_default(1024, 1024)
        P.lbm_submit(srv, big, np.ones((1024, 1024)), 10)
    assert ei.value.code == P.LBM_ERR_CAPACITY
    bad = np.full((40, 40), 1.0)
    bad[5, 5] = 8.5  # b rho > 1: psi undefined at once
    tb = P.lbm_submit(srv, P.lbm_desc_default(40, 40), bad, 50)
    good = [P.lbm_submit(srv, P.lbm_desc_default(120, 120, T=0.7),
                         synth.droplet(120, 120, 30.0, 0.7), 60 + 10 * k) for k in range(6)]
    res = wait(P, srv, good)
    assert all(r["rho"].shape == (120, 120) for r in res.values())
    t0 = time.time()
    while True:
        try:
            r = P.lbm_poll(srv, tb)
        except P.LbmError as e:
            assert e.code == P.LBM_ERR_NUMERIC
            break
        assert r is None and time.time() - t0 < 60
        time.sleep(0.002)
    with pytest.raises(P.LbmError) as ei:
        P.lbm_poll(srv, good[0])  # already collected
    assert ei.value.code == P.LBM_ERR_UNKNOWN_TICKET
    st = P.lbm_server_get_stats(srv)
    assert st["completed"] == 6 and st["failed"] == 1 and st["arena_in_use"] == 0
    P.lbm_server_destroy(srv)


def test_rho_only_results_without_velocity(P):
    # with_velocity = 0: results carry rho only (equal to the alone run); ux, uy are NaN
    opts = P.lbm_server_opts_default(arena_bytes=1 << 28, chunk_steps=25, with_velocity=0,
                                     kernel_variant=P.LBM_KERNEL_PLAIN, tile_x=TILE[0],
                                     tile_y=TILE[1])
    srv = P.lbm_server_create(opts)
    specs = [(64, 48, 14.0, 0.8, 60), (90, 90, 25.0, 0.7, 110), (40, 72, 10.0, 0.75, 35)]
    tickets, jobs = [], []
    for nx, ny, R, T, n in specs:
        d = P.lbm_desc_default(nx, ny, T=T)
        rho = synth.droplet(nx, ny, R, T)
        tickets.append(P.lbm_submit(srv, d, rho, n))
        jobs.append((d, rho, n))
    res = wait(P, srv, tickets)
    P.lbm_server_destroy(srv)
    for t, (d, rho, n) in zip(tickets, jobs):
        a = alone(P, d, rho, n)
        assert np.array_equal(res[t]["rho"], a["rho"])
        assert np.isnan(res[t]["ux"]).all() and np.isnan(res[t]["uy"]).all()


def test_tma_server_results_equal_plain_alone_runs(P):
    # the default server runs the single pass on the TMA kernel over its row
    # space (one tensor map for every resident lattice); its results equal
    # plain-kernel handles stepped alone, bitwise
    opts = P.lbm_server_opts_default(arena_bytes=1 << 30, chunk_steps=29, max_width=256)
    srv = P.lbm_server_create(opts)
    specs = [(200, 150, 40.0, 0.75, 130), (96, 96, 24.0, 0.65, 90), (130, 97, 30.0, 0.7, 61),
             (48, 40, 12.0, 0.8, 45), (256, 64, 20.0, 0.7, 70)]
    tickets, jobs = [], []
    for nx, ny, R, T, n in specs:
        d = P.lbm_desc_default(nx, ny, T=T)
        rho = synth.droplet(nx, ny, R, T)
        tickets.append(P.lbm_submit(srv, d, rho, n))
        jobs.append((d, rho, n))
    res = wait(P, srv, tickets)
    P.lbm_server_destroy(srv)
    for t, (d, rho, n) in zip(tickets, jobs):
        a = alone(P, d, rho, n)
        assert np.array_equal(res[t]["rho"], a["rho"]), (d.nx, d.ny)
        assert np.array_equal(res[t]["ux"], a["ux"])


def test_requests_in_turn_get_their_own_tables(P):
    # one request at a time, each polled before the next is submitted: a new
    # request then often occupies the memory of the one just polled, and the
    # server must still build its lattice table and tile lists (they are
    # reused only for the same tickets in the same order).  Shapes alternate
    # so that stale tables would step the wrong geometry.
    opts = P.lbm_server_opts_default(arena_bytes=1 << 28, chunk_steps=16,
                                     kernel_variant=P.LBM_KERNEL_PLAIN, tile_x=TILE[0],
                                     tile_y=TILE[1])
    srv = P.lbm_server_create(opts)
    shapes = [(40, 36, 10.0), (72, 30, 9.0), (33, 66, 10.0), (64, 64, 16.0)]
    for k in range(12):
        nx, ny, R = shapes[k % len(shapes)]
        d = P.lbm_desc_default(nx, ny, T=0.8)
        rho = synth.droplet(nx, ny, R, 0.8)
        n = 5 + 7 * k
        t = P.lbm_submit(srv, d, rho, n)
        r = wait(P, srv, [t])[t]
        a = alone(P, d, rho, n)
        assert np.array_equal(r["rho"], a["rho"]), (k, nx, ny)
        assert np.array_equal(r["ux"], a["ux"]), (k, nx, ny)
    st = P.lbm_server_get_stats(srv)
    assert st["completed"] == 12 and st["failed"] == 0
    P.lbm_server_destroy(srv)
