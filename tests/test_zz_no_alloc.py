"""The allocation-free mobility product against the handle-based one.

dbs_mobility_apply_noalloc serves callers that may not allocate device memory
while they run (a framework that owns all device memory through its own
capped pool, or a latency-critical loop where cudaMalloc would stall the
device).  Its scratch is one static array per GPU, shared by every call, so
this test makes two calls in a row -- the second smaller than the first, so
that stale scratch from the first call would show -- and checks each against
dbs_mobility_apply of a suspension handle with the same positions and forces,
within the FP32 pair-math tolerance of the parity tests (1e-5 of max |v|).
Further cases: the size limit itself (S = 4096, every scratch region full),
the smallest sizes (S = 1 and 8, one j-chunk), a suspension far from the
origin (the handle API re-centres; this entry point packs relative to its
first sphere), and an RPY overlap reported as DBS_E_OVERLAP followed by a
clean call (the status word is cleared for every call).
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


def _check_against_handle(S, x, F, s, mob):
    import torch
    with dbs.Suspension(x, a=s.a, mu=s.mu, k0=s.k0, ell=s.ell, omega=s.omega, dt=s.dt,
                        mobility=mob, precision="fp32c") as h:
        v_ref = h.mobility_apply(F)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    Fd = torch.from_numpy(np.ascontiguousarray(F)).cuda()
    vd = torch.full_like(xd, float("nan"))
    dbs.mobility_apply_noalloc(S, xd, Fd, a=s.a, mu=s.mu, mobility=mob, v_dev=vd)
    torch.cuda.synchronize()
    v = vd.cpu().numpy()
    assert np.isfinite(v).all()
    err = np.abs(v - v_ref).max() / np.abs(v_ref).max()
    assert err <= TOL, (S, err)
    return v


@pytest.mark.parametrize("S,mob", [(dbs.NOALLOC_MAX_S, "rpy"), (1, "rpy"), (8, "oseen"), (8, "rpy")])
def test_noalloc_edge_sizes(S, mob):
    import torch
    torch.cuda.set_device(0)
    if S <= 8:
        s = inputs.make_suspension(S, seed=21, side=8.0, mobility=mob)
    else:
        s = inputs.make_suspension(S, seed=22, density=0.002, mobility=mob)
    rng = np.random.default_rng(77 + S)
    F = rng.normal(size=s.x0.shape)
    _check_against_handle(S, s.x0, F, s, mob)


def test_noalloc_far_from_origin():
    import torch
    torch.cuda.set_device(0)
    s, x, F = _case(600, 5, "rpy")
    v0 = _check_against_handle(600, x, F, s, "rpy")
    shifted = x + np.array([500.0, -300.0, 800.0])
    v1 = _check_against_handle(600, shifted, F, s, "rpy")
    # the pair sum depends on differences only: the shift changes nothing beyond rounding
    assert np.abs(v1 - v0).max() / np.abs(v0).max() <= TOL


def test_noalloc_reports_overlap_then_recovers():
    import torch
    torch.cuda.set_device(0)
    s = inputs.make_suspension(8, seed=23, side=8.0, mobility="rpy")
    x = s.x0.copy()
    x[2] = x[0] + np.array([0.5 * s.a, 0.0, 0.0])     # two spheres closer than 2a
    F = np.random.default_rng(9).normal(size=x.shape)
    xd = torch.from_numpy(x).cuda()
    Fd = torch.from_numpy(F).cuda()
    vd = torch.zeros_like(xd)
    with pytest.raises(dbs.DbsError) as ei:
        dbs.mobility_apply_noalloc(8, xd, Fd, a=s.a, mu=s.mu, mobility="rpy", v_dev=vd)
    assert ei.value.status == dbs.E_OVERLAP
    # the next call on a valid geometry starts from a clear status word
    _check_against_handle(8, s.x0, F, s, "rpy")
