"""Host-side checks of the C-ABI library (no GPU needed).

* libdbs.so builds for sm_103a and loads, and exports every function that
  include/dbs.h declares.
* Argument validation happens before any CUDA call, so its error paths are
  exercised on the CPU: bad sizes, non-finite inputs, ell <= 2a (Sec. II
  requires ell > 2a + lambda), unknown enums.
* The seeded input generator is deterministic and honours its minimum separation.
"""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from paper_1004_1932_b300 import build, dbs, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return dbs.load()


def _declared():
    txt = open(os.path.join(ROOT, "include", "dbs.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(dbs_[a-z0-9_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 29, names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in dbs.h but not exported"


def test_status_strings(lib):
    assert dbs.status_string(dbs.OK) == "DBS_OK"
    assert dbs.status_string(dbs.E_OVERLAP) == "DBS_E_OVERLAP"
    assert lib.dbs_version().decode().startswith("dbs")


def _params(**kw):
    base = dict(S=2, a=0.05, mu=1.0, k0=1.0, ell=1.0, omega=2 * math.pi, dt=1e-3,
                mobility=dbs.RPY, precision=dbs.FP32C, stream=None, device=-1, flags=0)
    base.update(kw)
    return dbs.Params(**base)


@pytest.mark.parametrize("bad", [dict(S=0), dict(a=0.0), dict(mu=-1.0), dict(dt=0.0),
                                 dict(ell=0.1), dict(mobility=7), dict(precision=3),
                                 dict(flags=1), dict(omega=float("nan"))])
def test_create_rejects_bad_params(lib, bad):
    p = _params(**bad)
    x0 = np.zeros((2 * max(p.S, 1), 3))
    h = ctypes.c_void_p()
    rc = lib.dbs_create_suspension(ctypes.byref(p), x0.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   ctypes.byref(h))
    assert rc == dbs.E_ARG
    assert h.value is None
    assert len(lib.dbs_last_error(None)) > 0


def test_create_rejects_nonfinite_positions(lib):
    p = _params()
    x0 = np.zeros((4, 3))
    x0[2, 1] = np.inf
    h = ctypes.c_void_p()
    rc = lib.dbs_create_suspension(ctypes.byref(p), x0.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   ctypes.byref(h))
    assert rc == dbs.E_ARG


def test_sa_and_compare_reject_bad_sizes(lib):
    p = dbs.SaParams(1, 0.05, 1.0, 2 * math.pi, 0.01, dbs.K_PREFACTOR, dbs.FP32C, -1, None)
    z = np.zeros(3)
    h = ctypes.c_void_p()
    dp = ctypes.POINTER(ctypes.c_double)
    rc = lib.dbs_sa_create(ctypes.byref(p), z.ctypes.data_as(dp), z.ctypes.data_as(dp),
                           z.ctypes.data_as(dp), z.ctypes.data_as(dp), ctypes.byref(h))
    assert rc == dbs.E_ARG
    out = np.zeros(4)
    assert lib.dbs_pair_distance_error(ctypes.c_int64(1), None, None, None, None,
                                       out.ctypes.data_as(dp), None) == dbs.E_ARG
    assert lib.dbs_pair_distance_error_async(ctypes.c_int64(1), None, None, None, None, None,
                                             None) == dbs.E_ARG


def test_null_handles_are_rejected(lib):
    assert lib.dbs_step(None, ctypes.c_int64(1)) == dbs.E_ARG
    assert lib.dbs_sync(None) == dbs.E_ARG
    assert lib.dbs_destroy(None) == dbs.OK


def test_inputs_deterministic_and_separated():
    a = inputs.paper_scale(512, seed=3)
    b = inputs.paper_scale(512, seed=3)
    np.testing.assert_array_equal(a.x0, b.x0)
    d = np.linalg.norm(a.R0[:, None] - a.R0[None], axis=-1) + np.eye(512) * 1e9
    assert d.min() >= 2.0
    assert np.all(np.abs(a.R0) <= a.side / 2)
    np.testing.assert_allclose(np.linalg.norm(a.N0, axis=1), 1.0, rtol=1e-14)
    # spheres sit at their rest length at t = 0 (Sec. IV start)
    L0 = a.ell + a.lam * np.sin(a.phi)
    np.testing.assert_allclose(np.linalg.norm(a.x0[1::2] - a.x0[0::2], axis=1), L0, rtol=1e-13)
    assert a.side == pytest.approx((512 / 0.002) ** (1 / 3))


def test_engine_host_validation(lib):
    bad = dbs.EngineParams(0, 0, 0, -1, 0)            # block_steps must be >= 1
    h = ctypes.c_void_p()
    assert lib.dbs_engine_create(ctypes.byref(bad), ctypes.byref(h)) == dbs.E_ARG
    b1, b2 = dbs.request_bytes(100), dbs.request_bytes(1000)
    assert 0 < b1 < b2
    with pytest.raises(dbs.DbsError):
        dbs.request_bytes(0)
