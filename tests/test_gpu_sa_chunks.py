"""GPU parity of the source-chunked launch of the stroke-averaged model (Sec. III.B).

* With the sources of Eqs. (9a)-(9e) summed in C contiguous ranges by separate
  CTAs and merged in range order by the last CTA of each target group, the
  rates follow the FP64 oracle within the one-chunk tolerances (FP32C 1e-5,
  FP64 1e-12 of the largest rate) for chunk counts that do and do not fall on
  tile boundaries, with ragged last groups and ranges of a single source, and
  at the benchmark's size (S = 8192) and S = 12000 on the built-in split.
* Heun steps on the chunked launch follow the oracle's, two runs are
  bit-identical (the merge order does not depend on which CTA finishes last),
  and changing the count mid-run continues the same trajectory.
* The built-in count is 1 while the target groups fit one CTA per SM and the
  most even spread over the SMs above; a negative count is refused, 0 restores
  the built-in choice, and a count above S is clamped to S.
"""
import math

import numpy as np
import pytest
import torch
from scipy.spatial import cKDTree

import oracle
from paper_1004_1932_b300 import dbs, inputs

pytestmark = pytest.mark.gpu
TOL = {"fp32c": 1e-5, "fp64": 1e-12}


def _relerr(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def _sa(s, precision="fp32c", dt=0.1):
    h = dbs.StrokeAveraged(s.R0, s.N0, s.phi, s.lam, a=s.a, ell=s.ell, omega=s.omega, dt=dt,
                           precision=precision)
    h.set_path("grid")
    return h


def _kw(s):
    return dict(a=s.a, ell=s.ell, omega=s.omega)


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
@pytest.mark.parametrize("S,C", [(2, 2), (33, 5), (300, 2), (300, 7), (1000, 3), (2500, 4), (2500, 8), (5000, 3)])
def test_chunked_rates_match_oracle(S, C, prec):
    s = inputs.paper_scale(S, seed=40 + S + C)
    Rd_ref, Nd_ref = oracle.sa_rates(s.R0, s.N0, s.phi, s.lam, **_kw(s))
    with _sa(s, prec) as h:
        h.set_chunks(C)
        assert h.get_chunks() == min(C, S)
        Rd, Nd = h.rates()
    assert _relerr(Rd, Rd_ref) <= TOL[prec]
    assert _relerr(Nd, Nd_ref) <= TOL[prec]


@pytest.mark.parametrize("S", [8192, 12000])
def test_benchmark_size_rates_on_the_built_in_split(S):
    # the launch the benchmark times at S = 8192 (2 chunks) and a size whose
    # built-in count does not divide the tiles (12000: 4 chunks of 3000 sources)
    s = inputs.paper_scale(S, seed=5)
    Rd_ref, Nd_ref = oracle.sa_rates(s.R0, s.N0, s.phi, s.lam, **_kw(s))
    with _sa(s) as h:
        assert h.get_chunks() > 1
        Rd, Nd = h.rates()
    # at these sizes the FP32 rounding of the records' positions (relative to
    # the centre c of the bounding box) sets the error: one ulp of max|R - c| in
    # each coordinate of D, amplified 5x relatively by the D^-5 of the K term
    # at the closest pair
    c = 0.5 * (s.R0.min(0) + s.R0.max(0))
    dmin = cKDTree(s.R0).query(s.R0, k=2)[0][:, 1].min()
    tol = TOL["fp32c"] + 5 * math.sqrt(3) * float(np.spacing(np.float32(np.abs(s.R0 - c).max()))) / dmin
    assert _relerr(Rd, Rd_ref) <= tol
    assert _relerr(Nd, Nd_ref) <= tol


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
def test_chunked_steps_follow_oracle_and_repeat_bitwise(prec):
    s = inputs.paper_scale(3000, seed=7)
    nsteps = 40
    R_ref, N_ref = oracle.sa_heun(s.R0, s.N0, s.phi, s.lam, dt=0.1, nsteps=nsteps, **_kw(s))
    out = []
    for _ in range(2):
        with _sa(s, prec) as h:
            h.set_chunks(5)
            h.step(nsteps)
            out.append(h.state())
    (R, N), (R2, N2) = out
    assert np.array_equal(R, R2) and np.array_equal(N, N2)
    dR = np.abs(R_ref - s.R0).max()
    assert np.abs(R - R_ref).max() <= 10 * TOL[prec] * dR + 1e-13 * np.abs(R_ref).max()
    np.testing.assert_allclose(np.linalg.norm(N, axis=1), 1.0, rtol=1e-14)


def test_changing_the_count_mid_run_continues_the_trajectory():
    s = inputs.paper_scale(2500, seed=9)
    with _sa(s) as h:
        h.set_chunks(1)
        h.step(20)
        h.set_chunks(6)
        h.step(20)
        R, N = h.state()
    with _sa(s) as h:
        h.set_chunks(1)
        h.step(40)
        R1, N1 = h.state()
    dR = np.abs(R1 - s.R0).max()
    assert np.abs(R - R1).max() <= 10 * TOL["fp32c"] * dR + 1e-13 * np.abs(R1).max()


def _builtin(S, sms):
    # targets per CTA: grid within about 128 CTAs, at most 16, or 32 (FP32) once
    # groups of 32 outnumber the SMs
    tl_max = 32 if S > 32 * sms else 16
    tl = 1
    while tl < tl_max and S > 128 * tl:
        tl *= 2
    groups = -(-S // tl)
    if groups <= sms:
        return 1
    best, best_e = 1, -1.0
    for C in range(1, 9):
        u = groups * C / sms
        e = u / math.ceil(u) - 0.015 * (C - 1)
        if e > best_e + 1e-12:
            best, best_e = C, e
    return best


@pytest.mark.parametrize("S", [512, 2048, 3000, 8192])
def test_builtin_count_and_refusals(S):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    s = inputs.paper_scale(S, seed=1)
    with _sa(s) as h:
        assert h.get_chunks() == _builtin(S, sms)
        with pytest.raises(dbs.DbsError) as ei:
            h.set_chunks(-1)
        assert ei.value.status == dbs.E_ARG
        h.set_chunks(3)
        assert h.get_chunks() == 3
        h.set_chunks(0)
        assert h.get_chunks() == _builtin(S, sms)
        h.step(2)
        assert np.isfinite(h.state()[0]).all()
    tiny = inputs.paper_scale(2, seed=1)
    with _sa(tiny) as h:
        h.set_chunks(64)
        assert h.get_chunks() == 2
