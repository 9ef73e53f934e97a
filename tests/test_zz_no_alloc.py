"""GPU test of lbm_mass_noalloc, the mass sum that allocates nothing.

It is meant for callers that may not allocate device memory when they
check a mass (under an application's own up-front allocator, in a
real-time loop).  The test sums an FP32 density field with it and checks
the result against an exactly rounded sum of the same values (math.fsum)
and against the library's own mass reduction, lbm_mass, of a handle
initialised with that field.  It does so on two calls in a row with
different inputs (so a stale partial sum from the first call would show).
It lives in a file of its own that pytest collects last.
"""
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _case(P, torch, nx, ny, T, R):
    rho32 = synth.droplet(nx, ny, R, T).astype(np.float32)
    h = P.lbm_create(P.lbm_desc_default(nx, ny, T=T))
    P.lbm_init(h, 0, rho32.astype(np.float64))
    handle_mass = P.lbm_mass(h, 0)
    P.lbm_destroy(h)
    exact = math.fsum(rho32.astype(np.float64).ravel().tolist())
    return torch.from_numpy(rho32.reshape(-1)).cuda(), exact, handle_mass


def test_mass_noalloc_matches_lbm_mass_twice():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2003_07968_gb300 import build, capi as P

    build.build()
    P.load()
    stream = torch.cuda.current_stream()
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    a, exact_a, mass_a = _case(P, torch, 300, 257, 0.7, 60.0)
    b, exact_b, mass_b = _case(P, torch, 64, 48, 0.8, 12.0)  # fewer blocks than the first call
    P.lbm_mass_noalloc(a.data_ptr(), a.numel(), 0.0, out.data_ptr(), stream.cuda_stream)
    P.lbm_mass_noalloc(b.data_ptr(), b.numel(), 0.0, out.data_ptr() + 8, stream.cuda_stream)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    # the reduction itself: FP64 sums of FP32 values, against exact rounding
    assert abs(got[0] - exact_a) <= 1e-12 * exact_a
    assert abs(got[1] - exact_b) <= 1e-12 * exact_b
    # the handle stores the field as rest-referenced deviations whose mass
    # equals the field's up to the FP32 roundings of its small stored
    # differences (at most 2^-24 of their sum: below 1e-9 of the mass here)
    assert abs(got[0] - mass_a) <= 1e-9 * mass_a
    assert abs(got[1] - mass_b) <= 1e-9 * mass_b
    # an offset is added once
    P.lbm_mass_noalloc(b.data_ptr(), b.numel(), 2.5, out.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    assert abs(out[0].item() - (exact_b + 2.5)) <= 1e-12 * exact_b
    # sizes beyond the fixed scratch are refused before any GPU work
    with pytest.raises(P.LbmError) as ei:
        P.lbm_mass_noalloc(b.data_ptr(), P.LBM_NOALLOC_MAX_COUNT + 1, 0.0, out.data_ptr(),
                           stream.cuda_stream)
    assert ei.value.code == P.LBM_ERR_CAPACITY
