"""GPU test of lbm_mass_noalloc, the mass reduction that allocates nothing.

It is meant for callers that may not allocate device memory when they
check the conserved mass (inside a stream capture, under an application's
own up-front allocator, in a real-time loop).  The test feeds it the
populations that lbm_init writes for a lattice and checks its result
against the handle's own lbm_mass, on two calls in a row with different
inputs (so a stale partial sum from the first call would show).  It lives in
a file of its own that pytest collects last.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def _case(P, torch, nx, ny, T, R):
    rho = synth.droplet(nx, ny, R, T)
    # plain FP32 storage: the handle stores f_i = f_i^eq(rho, 0) = w_i rho
    # (rounded to FP32) at shifted sites, so the same multiset of values is
    # w_i rho rounded to FP32 over all sites and directions
    h = P.lbm_create(P.lbm_desc_default(nx, ny, T=T, storage=P.LBM_STORE_F32))
    P.lbm_init(h, 0, rho)
    want = P.lbm_mass(h, 0)
    P.lbm_destroy(h)
    vals = (W[:, None, None] * rho[None]).astype(np.float32)
    return torch.from_numpy(vals.reshape(-1)).cuda(), want


def test_mass_noalloc_matches_lbm_mass_twice():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2003_07968_gb300 import build, capi as P

    build.build()
    P.load()
    stream = torch.cuda.current_stream()
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    a, want_a = _case(P, torch, 300, 257, 0.7, 60.0)
    b, want_b = _case(P, torch, 64, 48, 0.8, 12.0)  # fewer blocks than the first call
    P.lbm_mass_noalloc(a.data_ptr(), a.numel(), 0.0, out.data_ptr(), stream.cuda_stream)
    P.lbm_mass_noalloc(b.data_ptr(), b.numel(), 0.0, out.data_ptr() + 8, stream.cuda_stream)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert abs(got[0] - want_a) <= 1e-12 * want_a
    assert abs(got[1] - want_b) <= 1e-12 * want_b
    # an offset is added once
    P.lbm_mass_noalloc(b.data_ptr(), b.numel(), 2.5, out.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    assert abs(out[0].item() - (want_b + 2.5)) <= 1e-12 * want_b
    # sizes beyond the fixed scratch are refused before any GPU work
    with pytest.raises(P.LbmError) as ei:
        P.lbm_mass_noalloc(b.data_ptr(), P.LBM_NOALLOC_MAX_COUNT + 1, 0.0, out.data_ptr(),
                           stream.cuda_stream)
    assert ei.value.code == P.LBM_ERR_CAPACITY
