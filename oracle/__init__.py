"""FP64 CPU oracle for the active-dumbbell hot path (TEST INFRASTRUCTURE ONLY).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library; the two meet only in the seeded inputs.

Functions (all float64 numpy, spheres 0-based, dumbbell s = spheres 2s, 2s+1):

=========================  ===================================================
``rest_length``            Eq. (4): L^s(t) = ell + lambda^s sin(omega t + phi^s)
``spring_forces``          Eq. (4): F = -dU/dX, U^s = k0/2 (d^s - L^s)^2
``mobility_apply``         Eq. (1a) at T=0 with Eq. (3): v = H F (self + pairs)
``interaction``            the pair part of Eq. (3b) alone
``mobility_matrix``        the dense 3N x 3N tensor of Eq. (3) (Sec. IV method)
``velocities``             spring (+ external) forces through Eq. (3)
``heun``                   Heun predictor-corrector, Sec. IV
``heun_period_avg``        Heun + stroke-averaged centres, Eqs. (6b), (7b)
``sa_rates`` / ``sa_heun`` stroke-averaged far-field EOM, Eqs. (9a)-(9e)
``pair_distance_change``   change of all pairwise centre distances
=========================  ===================================================

Parity pins live in ``tests/test_oracle_*.py``; ``shape_driven`` holds the
exact (not far-field-expanded) two-dumbbell shape-driven stroke average used
to pin the stroke-averaged law.
"""
import ctypes
import os

import numpy as np

from . import build as _build

OSEEN = 0
RPY = 1
K_PREFACTOR_PRINTED = 15.0 / 64.0  # Eq. (9d) as printed

_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_i64 = ctypes.c_int64


class _Params(ctypes.Structure):
    _fields_ = [("S", ctypes.c_int64), ("a", ctypes.c_double), ("mu", ctypes.c_double),
                ("k0", ctypes.c_double), ("ell", ctypes.c_double), ("omega", ctypes.c_double),
                ("dt", ctypes.c_double), ("mobility", ctypes.c_int)]


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
        _lib.orc_rest_length.restype = ctypes.c_double
        _lib.orc_rest_length.argtypes = [ctypes.c_double] * 5
    return _lib


def _c(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def set_threads(n: int) -> None:
    """Number of OpenMP threads the oracle uses (environment OMP_NUM_THREADS)."""
    os.environ["OMP_NUM_THREADS"] = str(int(n))
    try:
        ctypes.CDLL("libgomp.so.1").omp_set_num_threads(int(n))
    except OSError:
        pass


def rest_length(ell, lam, omega, phi, t):
    return lib().orc_rest_length(float(ell), float(lam), float(omega), float(phi), float(t))


def spring_forces(x, ell, lam, omega, phi, k0, t):
    x, px = _c(x)
    lam, pl = _c(lam)
    phi, pp = _c(phi)
    S = lam.shape[0]
    assert x.shape == (2 * S, 3)
    F = np.empty_like(x)
    lib().orc_spring_forces(_i64(S), px, ctypes.c_double(ell), pl, ctypes.c_double(omega), pp,
                            ctypes.c_double(k0), ctypes.c_double(t), F.ctypes.data_as(_dp))
    return F


def mobility_apply(x, F, a, mu, mobility=RPY):
    x, px = _c(x)
    F, pF = _c(F)
    v = np.empty_like(x)
    lib().orc_mobility_apply(_i64(x.shape[0]), px, pF, ctypes.c_double(a), ctypes.c_double(mu),
                             ctypes.c_int(mobility), v.ctypes.data_as(_dp))
    return v


def interaction(x, F, a, mu, mobility=RPY):
    x, px = _c(x)
    F, pF = _c(F)
    u = np.empty_like(x)
    lib().orc_interaction(_i64(x.shape[0]), px, pF, ctypes.c_double(a), ctypes.c_double(mu),
                          ctypes.c_int(mobility), u.ctypes.data_as(_dp))
    return u


def mobility_matrix(x, a, mu, mobility=RPY):
    x, px = _c(x)
    N = x.shape[0]
    H = np.empty((3 * N, 3 * N))
    lib().orc_mobility_matrix(_i64(N), px, ctypes.c_double(a), ctypes.c_double(mu),
                              ctypes.c_int(mobility), H.ctypes.data_as(_dp))
    return H


def _params(S, a, mu, k0, ell, omega, dt, mobility):
    return _Params(int(S), float(a), float(mu), float(k0), float(ell), float(omega), float(dt),
                   int(mobility))


def velocities(x, t, *, a, mu, k0, ell, omega, lam, phi, mobility=RPY, Fext=None):
    x, px = _c(x)
    lam, pl = _c(lam)
    phi, pp = _c(phi)
    p = _params(lam.shape[0], a, mu, k0, ell, omega, 0.0, mobility)
    pe = None
    if Fext is not None:
        Fext, pe = _c(Fext)
    v = np.empty_like(x)
    lib().orc_velocities(ctypes.byref(p), pl, pp, pe, px, ctypes.c_double(t), v.ctypes.data_as(_dp))
    return v


def heun(x, n0, nsteps, *, a, mu, k0, ell, omega, dt, lam, phi, mobility=RPY, Fext=None,
         kT=0.0, seed=0):
    """Advance positions ``x`` (copied) by ``nsteps`` Heun steps from step ``n0``;
    with kT > 0 the additive noise of ``orc_heun_noise`` (generator key ``seed``)."""
    x = np.array(x, dtype=np.float64, order="C", copy=True)
    lam, pl = _c(lam)
    phi, pp = _c(phi)
    p = _params(lam.shape[0], a, mu, k0, ell, omega, dt, mobility)
    pe = None
    if Fext is not None:
        Fext, pe = _c(Fext)
    if kT > 0:
        lib().orc_heun_noise(ctypes.byref(p), pl, pp, pe, x.ctypes.data_as(_dp), _i64(n0),
                             _i64(nsteps), ctypes.c_double(kT), ctypes.c_uint64(int(seed)))
    else:
        lib().orc_heun(ctypes.byref(p), pl, pp, pe, x.ctypes.data_as(_dp), _i64(n0), _i64(nsteps))
    return x


def sd_rates(x, t, niter, *, a, mu, k0=0.0, ell, omega, lam, phi, mobility=RPY):
    """Shape-driven model (Appendix A.2): (dR/dt [S,3], dN/dt [S,3], f [S]) at
    positions x and time t after ``niter`` constraint iterations."""
    x, px = _c(x)
    lam, pl = _c(lam)
    phi, pp = _c(phi)
    S = lam.shape[0]
    p = _params(S, a, mu, k0, ell, omega, 0.0, mobility)
    Rd, Nd, f = np.empty((S, 3)), np.empty((S, 3)), np.empty(S)
    lib().orc_sd_rates(ctypes.byref(p), pl, pp, px, ctypes.c_double(t), ctypes.c_int(int(niter)),
                       Rd.ctypes.data_as(_dp), Nd.ctypes.data_as(_dp), f.ctypes.data_as(_dp))
    return Rd, Nd, f


def sd_heun(x, n0, nsteps, niter, *, a, mu, k0=0.0, ell, omega, dt, lam, phi, mobility=RPY):
    """Heun on (R, N) of the shape-driven model; returns the sphere positions."""
    x = np.array(x, dtype=np.float64, order="C", copy=True)
    lam, pl = _c(lam)
    phi, pp = _c(phi)
    p = _params(lam.shape[0], a, mu, k0, ell, omega, dt, mobility)
    lib().orc_sd_heun(ctypes.byref(p), pl, pp, x.ctypes.data_as(_dp), _i64(n0), _i64(nsteps),
                      ctypes.c_int(int(niter)))
    return x


def philox4x32_10(ctr, key):
    """Philox4x32-10 on a 4-word counter with a 2-word key; returns 4 uint32."""
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def sphere_normals(seed, n, i):
    """The three standard normals of sphere i at step n (additive noise)."""
    z = np.empty(3)
    lib().orc_sphere_normals(ctypes.c_uint64(int(seed)), _i64(n), _i64(i), z.ctypes.data_as(_dp))
    return z


def heun_period_avg(x, n0, m, nper, *, a, mu, k0, ell, omega, dt, lam, phi, mobility=RPY,
                    Fext=None):
    """Heun over ``nper`` periods of ``m`` steps; returns (x_end, Rbar[nper, S, 3])."""
    x = np.array(x, dtype=np.float64, order="C", copy=True)
    lam, pl = _c(lam)
    phi, pp = _c(phi)
    S = lam.shape[0]
    p = _params(S, a, mu, k0, ell, omega, dt, mobility)
    Rbar = np.empty((nper, S, 3))
    pe = None
    if Fext is not None:
        Fext, pe = _c(Fext)
    lib().orc_heun_period_avg(ctypes.byref(p), pl, pp, pe, x.ctypes.data_as(_dp), _i64(n0), _i64(m),
                              _i64(nper), Rbar.ctypes.data_as(_dp))
    return x, Rbar


def sa_rates(R, Nv, phi, lam, *, a, ell, omega, kpref=K_PREFACTOR_PRINTED):
    R, pR = _c(R)
    Nv, pN = _c(Nv)
    phi, pp = _c(phi)
    lam, pl = _c(lam)
    Rdot = np.empty_like(R)
    Ndot = np.empty_like(Nv)
    lib().orc_sa_rates(_i64(R.shape[0]), pR, pN, pp, pl, ctypes.c_double(a), ctypes.c_double(ell),
                       ctypes.c_double(omega), ctypes.c_double(kpref), Rdot.ctypes.data_as(_dp),
                       Ndot.ctypes.data_as(_dp))
    return Rdot, Ndot


def sa_heun(R, Nv, phi, lam, *, a, ell, omega, dt, nsteps, kpref=K_PREFACTOR_PRINTED):
    R = np.array(R, dtype=np.float64, order="C", copy=True)
    Nv = np.array(Nv, dtype=np.float64, order="C", copy=True)
    phi, pp = _c(phi)
    lam, pl = _c(lam)
    lib().orc_sa_heun(_i64(R.shape[0]), R.ctypes.data_as(_dp), Nv.ctypes.data_as(_dp), pp, pl,
                      ctypes.c_double(a), ctypes.c_double(ell), ctypes.c_double(omega),
                      ctypes.c_double(kpref), ctypes.c_double(dt), _i64(nsteps))
    return R, Nv


def pair_distance_change(R0, R1):
    R0, p0 = _c(R0)
    R1, p1 = _c(R1)
    S = R0.shape[0]
    dD = np.empty((S, S))
    lib().orc_pair_distance_change(_i64(S), p0, p1, dD.ctypes.data_as(_dp))
    return dD


def pair_distance_error(dD_model, dD_ref):
    """max and RMS over pairs s<r of |dD_model - dD_ref|, and RMS|dD_ref|."""
    S = dD_ref.shape[0]
    iu = np.triu_indices(S, 1)
    e = np.abs(dD_model[iu] - dD_ref[iu])
    return {"max": float(e.max()), "rms": float(np.sqrt(np.mean(e * e))),
            "ref_rms": float(np.sqrt(np.mean(dD_ref[iu] ** 2)))}


def mobility_rows(x, F, rows, a, mu, mobility=RPY):
    """Eq. (3) evaluated only for the target spheres ``rows`` (int array)."""
    x, px = _c(x)
    F, pF = _c(F)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    v = np.empty((rows.shape[0], 3))
    lib().orc_mobility_rows(_i64(x.shape[0]), px, pF, ctypes.c_double(a), ctypes.c_double(mu),
                            ctypes.c_int(mobility), rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                            _i64(rows.shape[0]), v.ctypes.data_as(_dp))
    return v
