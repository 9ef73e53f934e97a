"""Failure detection for device allocations, injected on the host.

The library takes all device memory from the caller's allocator
(lbm_runtime_opts.alloc for handles, lbm_server_opts.alloc for the server).
An allocator that answers NULL on its k-th call stands in for an exhausted
device: for every k that a create makes, the create must return
LBM_ERR_OOM and give back everything it had taken (nothing stays
allocated), and a later create, init and step must work.  No GPU fault is
involved; the failure is an ordinary NULL from a host callback.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2003_07968_gb300 import build, capi

    build.build()
    capi.load()
    return capi


class FailingAllocator:
    """torch's caching allocator, but the call number `fail_at` (1-based)
    returns NULL; counts calls and keeps what is live."""

    def __init__(self, P, fail_at=0):
        import torch

        self.torch, self.fail_at, self.calls, self.live = torch, fail_at, 0, {}
        self.alloc = P.ALLOC_FN(self._alloc)
        self.free = P.FREE_FN(self._free)

    def _alloc(self, nbytes, _ctx):
        self.calls += 1
        if self.calls == self.fail_at:
            return None
        t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device="cuda")
        self.live[t.data_ptr()] = t
        return t.data_ptr()

    def _free(self, ptr, _nbytes, _ctx):
        assert self.live.pop(int(ptr), None) is not None, "free of memory it did not give"


def _desc(P):
    return P.lbm_desc_default(64, 48, T=0.8)


def test_handle_create_fails_cleanly_at_every_allocation(P):
    probe = FailingAllocator(P)
    h = P.lbm_create(_desc(P), allocator=probe)
    n = probe.calls
    P.lbm_destroy(h)
    assert n >= 5 and not probe.live
    for k in range(1, n + 1):
        a = FailingAllocator(P, fail_at=k)
        with pytest.raises(P.LbmError) as ei:
            P.lbm_create(_desc(P), allocator=a)
        assert ei.value.code == P.LBM_ERR_OOM, k
        assert not a.live, f"allocation {k} of {n}: {len(a.live)} blocks left"
    # the next create, with an allocator that does not fail, works
    rho = synth.droplet(64, 48, 12.0, 0.8)
    h = P.lbm_create(_desc(P))
    P.lbm_init(h, 0, rho)
    P.lbm_step(h, 50)
    got = P.lbm_moments(h, 0, u=False)
    P.lbm_destroy(h)
    want = oracle.run(oracle.params(T=0.8), rho, 50)["rho"]
    assert float(np.max(np.abs(got["rho"] - want) / want)) <= 1e-5


def test_init_staging_allocation_failure_leaves_the_handle_usable(P):
    probe = FailingAllocator(P)
    h = P.lbm_create(_desc(P), allocator=probe)
    P.lbm_destroy(h)
    first_init_alloc = probe.calls + 1  # lbm_init's staging buffer comes next
    a = FailingAllocator(P, fail_at=first_init_alloc)
    h = P.lbm_create(_desc(P), allocator=a)
    rho = synth.droplet(64, 48, 12.0, 0.8)
    with pytest.raises(P.LbmError) as ei:
        P.lbm_init(h, 0, rho)
    assert ei.value.code == P.LBM_ERR_OOM
    P.lbm_init(h, 0, rho)  # the allocator answers again
    P.lbm_step(h, 20)
    got = P.lbm_moments(h, 0, u=False, mass=False)["rho"]
    P.lbm_destroy(h)
    assert not a.live
    want = oracle.run(oracle.params(T=0.8), rho, 20)["rho"]
    assert float(np.max(np.abs(got - want) / want)) <= 1e-5


def test_server_create_fails_cleanly_at_every_allocation(P):
    def opts(alloc):
        o = P.lbm_server_opts_default(arena_bytes=64 << 20, max_resident=16,
                                      max_request_sites=128 * 128, max_width=256)
        o.alloc, o.free, o.alloc_ctx = alloc.alloc, alloc.free, None
        return o

    probe = FailingAllocator(P)
    srv = P.lbm_server_create(opts(probe))
    n = probe.calls
    P.lbm_server_destroy(srv)
    assert n >= 5 and not probe.live
    for k in range(1, n + 1):
        a = FailingAllocator(P, fail_at=k)
        with pytest.raises(P.LbmError) as ei:
            P.lbm_server_create(opts(a))
        assert ei.value.code == P.LBM_ERR_OOM, k
        assert not a.live, f"allocation {k} of {n}: {len(a.live)} blocks left"
    # a server whose allocator answers serves a request
    good = FailingAllocator(P)
    srv = P.lbm_server_create(opts(good))
    rho = synth.droplet(64, 48, 12.0, 0.8)
    t = P.lbm_submit(srv, _desc(P), rho, 40)
    import time

    t0, res = time.time(), None
    while res is None:
        res = P.lbm_poll(srv, t, u=False)
        assert time.time() - t0 < 60
        time.sleep(0.002)
    P.lbm_server_destroy(srv)
    assert not good.live
    want = oracle.run(oracle.params(T=0.8), rho, 40)["rho"]
    assert float(np.max(np.abs(res["rho"] - want) / want)) <= 1e-5
