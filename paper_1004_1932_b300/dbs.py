"""ctypes binding of ``libdbs.so`` (C-ABI declared in ``include/dbs.h``).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Host arrays are float64 numpy arrays in the layouts of the header
([N][3] sphere-major, [S] per dumbbell); ``*_device`` calls take torch CUDA
tensors (or raw device pointers) and stay stream-ordered.

There is no fallback: if the library is missing or fails to load, ``load()``
raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdbs.so")

OK = 0
E_ARG, E_NOMEM, E_CUDA, E_OVERLAP, E_NONFINITE, E_TIMEOUT, E_STATE = -1, -2, -3, -4, -5, -6, -7
OSEEN, RPY = 0, 1
FP32C, FP64 = 0, 1
PATH_GRID, PATH_CLUSTER, PATH_COOP = 0, 1, 2
_PATHS = {"grid": PATH_GRID, "cluster": PATH_CLUSTER, "coop": PATH_COOP}
K_PREFACTOR = 15.0 / 64.0  # Eq. (9d) as printed

_dp = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64


class Params(ctypes.Structure):
    _fields_ = [("S", ctypes.c_int64), ("a", ctypes.c_double), ("mu", ctypes.c_double),
                ("k0", ctypes.c_double), ("ell", ctypes.c_double), ("omega", ctypes.c_double),
                ("dt", ctypes.c_double), ("mobility", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("stream", ctypes.c_void_p),
                ("device", ctypes.c_int32), ("flags", ctypes.c_int32)]


class SaParams(ctypes.Structure):
    _fields_ = [("S", ctypes.c_int64), ("a", ctypes.c_double), ("ell", ctypes.c_double),
                ("omega", ctypes.c_double), ("dt", ctypes.c_double), ("kpref", ctypes.c_double),
                ("precision", ctypes.c_int32), ("device", ctypes.c_int32),
                ("stream", ctypes.c_void_p)]


class DbsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{status_string(status)}: {msg}")
        self.status = status


_lib = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libdbs.so (raises OSError/FileNotFoundError if it is absent)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise FileNotFoundError(f"{p} not built; run python -m paper_1004_1932_b300.build")
    lib = ctypes.CDLL(p)
    for name in ("dbs_last_error", "dbs_status_string", "dbs_version", "dbs_sa_last_error",
                 "dbs_ensemble_last_error", "dbs_engine_last_error"):
        getattr(lib, name).restype = ctypes.c_char_p
    lib.dbs_last_error.argtypes = [_vp]
    lib.dbs_sa_last_error.argtypes = [_vp]
    lib.dbs_ensemble_last_error.argtypes = [_vp]
    lib.dbs_engine_last_error.argtypes = [_vp]
    lib.dbs_status_string.argtypes = [ctypes.c_int]
    _lib = lib
    return lib


def status_string(s: int) -> str:
    return load().dbs_status_string(int(s)).decode()


def _arr(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.shape != tuple(shape):
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


def _p(a):
    return a.ctypes.data_as(_dp)


def _devptr(t) -> int:
    return int(t.data_ptr()) if hasattr(t, "data_ptr") else int(t)


def _mob(m):
    if isinstance(m, str):
        return {"oseen": OSEEN, "rpy": RPY}[m.lower()]
    return int(m)


def _prec(p):
    if isinstance(p, str):
        return {"fp32c": FP32C, "fp64": FP64}[p.lower()]
    return int(p)


class Suspension:
    """One simulated suspension (handle of ``dbs_create_suspension``)."""

    def __init__(self, x0, *, a, mu, k0, ell, omega, dt, mobility="rpy", precision="fp32c",
                 lam=None, phi=None, stream=None, device=-1):
        lib = load()
        x0 = _arr(x0)
        if x0.ndim != 2 or x0.shape[1] != 3 or x0.shape[0] % 2:
            raise ValueError("x0 must be [2S, 3]")
        self.S = x0.shape[0] // 2
        self.N = 2 * self.S
        self._p = Params(self.S, a, mu, k0, ell, omega, dt, _mob(mobility), _prec(precision),
                         stream if stream is None else ctypes.c_void_p(_devptr_stream(stream)),
                         device, 0)
        h = ctypes.c_void_p()
        rc = lib.dbs_create_suspension(ctypes.byref(self._p), _p(x0), ctypes.byref(h))
        if rc != OK:
            raise DbsError(rc, lib.dbs_last_error(None).decode())
        self._h = h
        if lam is not None or phi is not None:
            self.set_stroke(np.zeros(self.S) if lam is None else lam,
                            np.zeros(self.S) if phi is None else phi)

    @classmethod
    def from_inputs(cls, susp, precision="fp32c", mobility=None, **kw):
        """Create from a ``paper_1004_1932_b300.inputs.Suspension``."""
        return cls(susp.x0, a=susp.a, mu=susp.mu, k0=susp.k0, ell=susp.ell, omega=susp.omega,
                   dt=susp.dt, mobility=mobility or susp.mobility, precision=precision,
                   lam=susp.lam, phi=susp.phi, **kw)

    # -- plumbing --------------------------------------------------------
    def _check(self, rc):
        if rc != OK:
            raise DbsError(rc, load().dbs_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            load().dbs_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- ABI mirror ----------------------------------------------------------
    def set_stroke(self, lam, phi):
        lam = _arr(np.broadcast_to(np.asarray(lam, float), (self.S,)))
        phi = _arr(phi, (self.S,))
        self._check(load().dbs_set_stroke(self._h, _p(lam), _p(phi)))

    def set_external_force(self, F):
        if F is None:
            self._check(load().dbs_set_external_force(self._h, None))
        else:
            F = _arr(F, (self.N, 3))
            self._check(load().dbs_set_external_force(self._h, _p(F)))

    def set_dynamics(self, model: str = "spring", iterations: int = 2):
        """"spring" (Eq. (4), default) or "shape": shape-driven dumbbells, lengths
        held at L(t) by ``iterations`` steps of the constraint-force iteration."""
        m = {"spring": 0, "shape": 1}[model]
        self._check(load().dbs_set_dynamics(self._h, ctypes.c_int32(m), ctypes.c_int32(int(iterations))))

    def set_flow_tag(self, tag: int):
        """Diagnostic: the next evaluation tag of the cooperative path (wrap-around tests)."""
        self._check(load().dbs_test_set_flow_tag(self._h, ctypes.c_uint32(int(tag))))

    def set_noise(self, kT: float, seed: int = 0):
        """Additive Brownian noise of temperature kT (0 = off), generator key ``seed``."""
        self._check(load().dbs_set_noise(self._h, ctypes.c_double(float(kT)),
                                         ctypes.c_uint64(int(seed) & 0xFFFFFFFFFFFFFFFF)))

    def step(self, n: int = 1):
        self._check(load().dbs_step(self._h, _i64(int(n))))

    def sync(self):
        self._check(load().dbs_sync(self._h))

    def velocities(self):
        v = np.empty((self.N, 3))
        self._check(load().dbs_velocities(self._h, _p(v)))
        return v

    def interaction(self):
        u = np.empty((self.N, 3))
        self._check(load().dbs_interaction(self._h, _p(u)))
        return u

    def mobility_apply(self, F):
        F = _arr(F, (self.N, 3))
        v = np.empty((self.N, 3))
        self._check(load().dbs_mobility_apply(self._h, _p(F), _p(v)))
        return v

    def velocities_device(self, out):
        """Velocities at the current state into a device tensor ``out`` ([N, 3] float64)."""
        self._check(load().dbs_velocities_device(self._h, ctypes.c_void_p(_devptr(out))))

    def step_timed(self, n: int) -> float:
        """n Heun steps one launch at a time; returns mean ms per pair-sum launch."""
        ms = ctypes.c_double()
        self._check(load().dbs_step_timed(self._h, _i64(int(n)), ctypes.byref(ms)))
        return ms.value

    def set_path(self, path, cluster_size: int = 0):
        """dbs_step path: "grid" (per-evaluation launches), "cluster" (resident
        cluster) or "coop" (one cooperative launch per up to 1024 steps)."""
        p = _PATHS.get(path, path)
        self._check(load().dbs_set_path(self._h, ctypes.c_int32(int(p)), ctypes.c_int32(int(cluster_size))))

    def get_path(self):
        p, g = ctypes.c_int32(), ctypes.c_int32()
        self._check(load().dbs_get_path(self._h, ctypes.byref(p), ctypes.byref(g)))
        return {v: k for k, v in _PATHS.items()}[p.value], g.value

    def set_chunks(self, chunks: int):
        """j-split of the pair sum (0 = built-in choice); used by the autotuner."""
        self._check(load().dbs_set_chunks(self._h, ctypes.c_int32(int(chunks))))

    # -- row sharding (dbs_shard_*): one suspension split over several ranks --
    def shard_set(self, nranks: int, rank: int):
        """Compute only rank ``rank``'s row block in shard_eval; returns (row0, row1)."""
        r0, r1 = ctypes.c_int64(), ctypes.c_int64()
        self._check(load().dbs_shard_set(self._h, ctypes.c_int32(int(nranks)), ctypes.c_int32(int(rank)),
                                         ctypes.byref(r0), ctypes.byref(r1)))
        return r0.value, r1.value

    def shard_eval(self, phase: int):
        """One evaluation of the row block: 0 = predictor, 1 = corrector."""
        self._check(load().dbs_shard_eval(self._h, ctypes.c_int32(int(phase))))

    def shard_buffers(self):
        """(device pointer of record buffer A, of B, bytes per record)."""
        a, b, rb = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_int64()
        self._check(load().dbs_shard_buffers(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(rb)))
        return a.value, b.value, rb.value

    def get_launch(self):
        bt, c, g = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        self._check(load().dbs_get_launch(self._h, ctypes.byref(bt), ctypes.byref(c), ctypes.byref(g)))
        return {"bt": bt.value, "chunks": c.value, "grid": g.value}

    def positions(self):
        x = np.empty((self.N, 3))
        self._check(load().dbs_positions(self._h, _p(x)))
        return x

    def positions_device(self, out):
        """Copy positions into a device tensor ``out`` (float64, [N, 3])."""
        self._check(load().dbs_positions_device(self._h, ctypes.c_void_p(_devptr(out))))

    def get_time(self):
        n = ctypes.c_int64()
        t = ctypes.c_double()
        self._check(load().dbs_get_time(self._h, ctypes.byref(n), ctypes.byref(t)))
        return n.value, t.value

    def get_state(self):
        x = np.empty((self.N, 3))
        n = ctypes.c_int64()
        self._check(load().dbs_get_state(self._h, _p(x), ctypes.byref(n)))
        return x, n.value

    def set_state(self, x, n):
        x = _arr(x, (self.N, 3))
        self._check(load().dbs_set_state(self._h, _p(x), _i64(int(n))))

    def enable_period_average(self, m: int, max_periods: int = 64):
        self._check(load().dbs_enable_period_average(self._h, _i64(int(m)), _i64(int(max_periods))))

    def period_count(self) -> int:
        c = ctypes.c_int64()
        self._check(load().dbs_period_count(self._h, ctypes.byref(c)))
        return c.value

    def period_averages(self, k0: int = 0, count: int | None = None):
        if count is None:
            count = self.period_count() - k0
        R = np.empty((count, self.S, 3))
        self._check(load().dbs_period_averages(self._h, _i64(k0), _i64(count), _p(R)))
        return R

    def period_average_device(self, k: int) -> int:
        ptr = ctypes.c_void_p()
        self._check(load().dbs_period_average_device(self._h, _i64(k), ctypes.byref(ptr)))
        return ptr.value


def _devptr_stream(stream) -> int:
    if hasattr(stream, "cuda_stream"):
        return int(stream.cuda_stream)
    return int(stream)


class StrokeAveraged:
    """Stroke-averaged far-field model (handle of ``dbs_sa_create``)."""

    def __init__(self, R, N, phi, lam, *, a, ell, omega, dt, kpref=K_PREFACTOR,
                 precision="fp32c", stream=None, device=-1):
        lib = load()
        R = _arr(R)
        self.S = R.shape[0]
        N = _arr(N, (self.S, 3))
        phi = _arr(phi, (self.S,))
        lam = _arr(np.broadcast_to(np.asarray(lam, float), (self.S,)))
        self._p = SaParams(self.S, a, ell, omega, dt, kpref, _prec(precision), device,
                           None if stream is None else ctypes.c_void_p(_devptr_stream(stream)))
        h = ctypes.c_void_p()
        rc = lib.dbs_sa_create(ctypes.byref(self._p), _p(R), _p(N), _p(phi), _p(lam), ctypes.byref(h))
        if rc != OK:
            raise DbsError(rc, lib.dbs_sa_last_error(None).decode())
        self._h = h

    def _check(self, rc):
        if rc != OK:
            raise DbsError(rc, load().dbs_sa_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            load().dbs_sa_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1):
        self._check(load().dbs_sa_step(self._h, _i64(int(n))))

    def set_path(self, path: str):
        """"grid" (one launch per evaluation) or "coop" (FP32C, S <= 4096; the default there)."""
        self._check(load().dbs_sa_set_path(self._h, ctypes.c_int32(_PATHS[path])))

    def get_path(self):
        p, t = ctypes.c_int32(), ctypes.c_int32()
        self._check(load().dbs_sa_get_path(self._h, ctypes.byref(p), ctypes.byref(t)))
        return {v: k for k, v in _PATHS.items()}[p.value], t.value

    def set_chunks(self, chunks: int):
        """Source chunks of the "grid" path's launch (0: the built-in choice)."""
        self._check(load().dbs_sa_set_chunks(self._h, ctypes.c_int32(int(chunks))))

    def get_chunks(self) -> int:
        c = ctypes.c_int32()
        self._check(load().dbs_sa_get_chunks(self._h, ctypes.byref(c)))
        return c.value

    def rates(self):
        Rd = np.empty((self.S, 3))
        Nd = np.empty((self.S, 3))
        self._check(load().dbs_sa_rates(self._h, _p(Rd), _p(Nd)))
        return Rd, Nd

    def state(self):
        R = np.empty((self.S, 3))
        N = np.empty((self.S, 3))
        self._check(load().dbs_sa_state(self._h, _p(R), _p(N)))
        return R, N

    def copy_centres(self, out):
        """Stream-ordered copy of the centres into a device tensor ``out`` ([S, 3] float64)."""
        self._check(load().dbs_sa_copy_centres(self._h, ctypes.c_void_p(_devptr(out))))

    def centres_device(self) -> int:
        ptr = ctypes.c_void_p()
        self._check(load().dbs_sa_centres_device(self._h, ctypes.byref(ptr)))
        return ptr.value


def pair_distance_error(S, A0, A1, B0, B1, stream=None):
    """max and RMS of |dA - dB| over pairs, and RMS of dB (device pointers or tensors)."""
    out = np.empty(4)
    rc = load().dbs_pair_distance_error(
        _i64(int(S)), *(ctypes.c_void_p(_devptr(t)) for t in (A0, A1, B0, B1)), _p(out),
        None if stream is None else ctypes.c_void_p(_devptr_stream(stream)))
    if rc != OK:
        raise DbsError(rc, "dbs_pair_distance_error")
    return {"max": float(out[0]), "rms": float(out[1]), "ref_rms": float(out[2]), "pairs": int(out[3])}


def pair_distance_error_async(S, A0, A1, B0, B1, out, stream=None):
    """The same four values (max, RMS, RMS of dB, pairs) into ``out``, a device
    tensor of 4 doubles, enqueued on ``stream`` without synchronising."""
    rc = load().dbs_pair_distance_error_async(
        _i64(int(S)), *(ctypes.c_void_p(_devptr(t)) for t in (A0, A1, B0, B1, out)),
        None if stream is None else ctypes.c_void_p(_devptr_stream(stream)))
    if rc != OK:
        raise DbsError(rc, "dbs_pair_distance_error_async")


class Ensemble:
    """Independent suspensions advanced together on thread-block clusters
    (``dbs_ensemble_*``).  Members stay usable as ordinary handles."""

    def __init__(self, members, stream=None):
        lib = load()
        self.members = list(members)
        arr = (ctypes.c_void_p * len(self.members))(*[m._h.value for m in self.members])
        h = ctypes.c_void_p()
        rc = lib.dbs_ensemble_create(ctypes.c_int32(len(self.members)), arr,
                                     None if stream is None else ctypes.c_void_p(_devptr_stream(stream)),
                                     ctypes.byref(h))
        if rc != OK:
            raise DbsError(rc, lib.dbs_ensemble_last_error(None).decode())
        self._h = h

    def _check(self, rc):
        if rc != OK:
            raise DbsError(rc, load().dbs_ensemble_last_error(self._h).decode())

    def step(self, n: int = 1):
        self._check(load().dbs_ensemble_step(self._h, _i64(int(n))))

    def sync(self):
        self._check(load().dbs_ensemble_sync(self._h))

    def set_clusters(self, G=None):
        if G is None:
            self._check(load().dbs_ensemble_set_clusters(self._h, None))
        else:
            g = (ctypes.c_int32 * len(self.members))(*[int(x) for x in G])
            self._check(load().dbs_ensemble_set_clusters(self._h, g))

    def get_clusters(self):
        g = (ctypes.c_int32 * len(self.members))()
        self._check(load().dbs_ensemble_get_clusters(self._h, g))
        return list(g)

    def close(self):
        if getattr(self, "_h", None):
            load().dbs_ensemble_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


REQ_PENDING, REQ_RUNNING, REQ_DONE, REQ_CANCELLED, REQ_FAILED = 0, 1, 2, 3, 4


class EngineParams(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_active", ctypes.c_int32),
                ("block_steps", ctypes.c_int32), ("device", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class Engine:
    """Serving engine (``dbs_engine_*``): requests admitted by a device-memory
    budget and advanced together on every ``tick()`` (continuous batching)."""

    def __init__(self, hbm_budget_bytes: int = 0, max_active: int = 0, block_steps: int = 256,
                 device: int = -1):
        lib = load()
        self._p = EngineParams(int(hbm_budget_bytes), int(max_active), int(block_steps), int(device), 0)
        h = ctypes.c_void_p()
        rc = lib.dbs_engine_create(ctypes.byref(self._p), ctypes.byref(h))
        if rc != OK:
            raise DbsError(rc, lib.dbs_engine_last_error(None).decode())
        self._h = h
        self._S = {}

    def _check(self, rc):
        if rc != OK:
            raise DbsError(rc, load().dbs_engine_last_error(self._h).decode())

    def submit(self, x0, *, a, mu, k0, ell, omega, dt, steps, mobility="rpy", precision="fp32c",
               lam=None, phi=None) -> int:
        x0 = _arr(x0)
        S = x0.shape[0] // 2
        p = Params(S, a, mu, k0, ell, omega, dt, _mob(mobility), _prec(precision), None, -1, 0)
        lam_a = None if lam is None else _arr(np.broadcast_to(np.asarray(lam, float), (S,)))
        phi_a = None if phi is None else _arr(phi, (S,))
        rid = ctypes.c_int64()
        self._check(load().dbs_engine_submit(self._h, ctypes.byref(p), _p(x0),
                                             None if lam_a is None else _p(lam_a),
                                             None if phi_a is None else _p(phi_a),
                                             _i64(int(steps)), ctypes.byref(rid)))
        self._S[rid.value] = S
        return rid.value

    def submit_inputs(self, susp, steps, precision="fp32c") -> int:
        return self.submit(susp.x0, a=susp.a, mu=susp.mu, k0=susp.k0, ell=susp.ell, omega=susp.omega,
                           dt=susp.dt, steps=steps, mobility=susp.mobility, precision=precision,
                           lam=susp.lam, phi=susp.phi)

    def tick(self):
        a, q = ctypes.c_int32(), ctypes.c_int32()
        self._check(load().dbs_engine_tick(self._h, ctypes.byref(a), ctypes.byref(q)))
        return a.value, q.value

    def stats(self) -> dict:
        """Host-side accounting (``dbs_engine_stats``)."""
        class _St(ctypes.Structure):
            _fields_ = [("ticks", ctypes.c_int64), ("ensemble_rebuilds", ctypes.c_int64),
                        ("tick_s", ctypes.c_double), ("rebuild_s", ctypes.c_double),
                        ("wait_s", ctypes.c_double)]
        st = _St()
        self._check(load().dbs_engine_stats(self._h, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in _St._fields_}

    def poll(self, rid: int):
        st = ctypes.c_int32()
        x = np.empty((2 * self._S[rid], 3))
        lat = ctypes.c_double(float("nan"))
        self._check(load().dbs_engine_poll(self._h, _i64(rid), ctypes.byref(st), _p(x),
                                           ctypes.byref(lat)))
        return st.value, (x if st.value == REQ_DONE else None), lat.value

    def cancel(self, rid: int):
        self._check(load().dbs_engine_cancel(self._h, _i64(rid)))

    def close(self):
        if getattr(self, "_h", None):
            load().dbs_engine_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def request_bytes(S: int, precision="fp32c") -> int:
    b = ctypes.c_size_t()
    rc = load().dbs_engine_request_bytes(_i64(int(S)), ctypes.c_int32(_prec(precision)), ctypes.byref(b))
    if rc != OK:
        raise DbsError(rc, "dbs_engine_request_bytes")
    return b.value


NOALLOC_MAX_S = 4096


def mobility_apply_noalloc(S, x_dev, F_dev, *, a, mu, mobility="rpy", v_dev, stream=None):
    """v = H F on caller-owned device buffers without any allocation
    (``dbs_mobility_apply_noalloc``): for callers that may not allocate device
    memory while they run.  Shares one static scratch array per GPU; serialise
    overlapping calls."""
    rc = load().dbs_mobility_apply_noalloc(
        _i64(int(S)), ctypes.c_void_p(_devptr(x_dev)), ctypes.c_void_p(_devptr(F_dev)),
        ctypes.c_double(a), ctypes.c_double(mu), ctypes.c_int32(_mob(mobility)),
        ctypes.c_void_p(_devptr(v_dev)),
        None if stream is None else ctypes.c_void_p(_devptr_stream(stream)))
    if rc != OK:
        raise DbsError(rc, "dbs_mobility_apply_noalloc")


def check_wait_timeout(timeout_ms: int = 100) -> int:
    """Run the cooperative path's bounded wait on a word that nothing writes;
    returns the status it reported (E_TIMEOUT expected).  Raises if the device
    did not stay usable."""
    st = ctypes.c_int32(-100)
    rc = load().dbs_test_wait_timeout(ctypes.c_int32(int(timeout_ms)), ctypes.byref(st))
    if rc != OK:
        raise DbsError(rc, "dbs_test_wait_timeout")
    return st.value


class DeviceView:
    """Zero-copy view of library-owned device memory for torch (``torch.as_tensor``)."""

    def __init__(self, ptr: int, shape, device_index: int = 0, typestr: str = "<f8"):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3, "strides": None}
        self.device_index = device_index
