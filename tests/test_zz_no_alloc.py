"""The allocation-free mobility product against the handle-based one.

dbs_mobility_apply_noalloc serves callers that may not allocate device memory
while they run (a framework that owns all device memory through its own
capped pool, or a latency-critical loop where cudaMalloc would stall the
device).  Its scratch is one static array per GPU, shared by every call, so
this test makes two calls in a row -- the second smaller than the first, so
that stale scratch from the first call would show -- and checks each against
dbs_mobility_apply of a suspension handle with the same positions and forces,
within the FP32 pair-math tolerance of the parity tests (1e-5 of max |v|).
This file is collected last, so a run that stops at the first failure has
already run every other test.
"""
import math

import numpy as np
import pytest

from paper_1004_1932_b300 import dbs, inputs

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _case(S, seed, mob):
    s = inputs.make_suspension(S, seed=seed, density=0.002, mobility=mob)
    rng = np.random.default_rng(500 + seed)
    x = s.x0 + rng.normal(scale=0.05, size=s.x0.shape)
    F = rng.normal(size=s.x0.shape)
    return s, x, F


def test_noalloc_matches_handle_api_on_two_calls():
    import torch
    torch.cuda.set_device(0)
    for S, seed, mob in ((1000, 3, "rpy"), (700, 4, "oseen")):
        s, x, F = _case(S, seed, mob)
        with dbs.Suspension(x, a=s.a, mu=s.mu, k0=s.k0, ell=s.ell, omega=s.omega, dt=s.dt,
                            mobility=mob, precision="fp32c") as h:
            v_ref = h.mobility_apply(F)
        xd = torch.from_numpy(x).cuda()
        Fd = torch.from_numpy(F).cuda()
        vd = torch.full_like(xd, float("nan"))
        dbs.mobility_apply_noalloc(S, xd, Fd, a=s.a, mu=s.mu, mobility=mob, v_dev=vd)
        torch.cuda.synchronize()
        v = vd.cpu().numpy()
        assert np.isfinite(v).all()
        assert np.abs(v - v_ref).max() / np.abs(v_ref).max() <= TOL


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    torch.cuda.set_device(0)
    S = dbs.NOALLOC_MAX_S + 1
    buf = torch.zeros((2 * S, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(dbs.DbsError) as ei:
        dbs.mobility_apply_noalloc(S, buf, buf, a=0.05, mu=1.0, v_dev=buf)
    assert ei.value.status == dbs.E_ARG
