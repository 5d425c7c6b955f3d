"""Seeded synthetic inputs for active-dumbbell suspensions.

This module only draws random numbers and lays out initial conditions; it
holds none of the method's arithmetic (no forces, mobilities, integrators or
stroke averages).  Both the CUDA library's tests and the CPU oracle read the
arrays it returns, so every comparison starts from bit-identical inputs.

Initial condition (Sec. IV of the paper: each sphere starts at the minimum of
its spring potential, i.e. the dumbbell length equals its rest length at t=0):

* centres R^s uniform in the cube [-side/2, side/2]^3, drawn in index order
  and rejected while closer than ``min_sep`` to an accepted centre;
* orientations N^s uniform on the unit sphere (z ~ U(-1, 1), azimuth ~ U(0, 2pi));
* phases phi^s ~ U(0, 2pi) (or given);
* spheres 2s and 2s+1 at R^s -/+ N^s L^s(0) / 2 with L^s(0) = ell + lambda^s sin(phi^s),
  so N^s points from sphere 2s to sphere 2s+1.

All draws come from ``numpy.random.default_rng(seed)`` in the order
centres, orientations, phases.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Suspension:
    """One seeded suspension: physical parameters plus its initial state."""
    S: int
    a: float
    mu: float
    k0: float
    ell: float
    omega: float
    dt: float
    mobility: str              # "oseen" or "rpy"
    lam: np.ndarray            # [S] stroke amplitudes
    phi: np.ndarray            # [S] stroke phases
    R0: np.ndarray             # [S, 3] centres
    N0: np.ndarray             # [S, 3] unit orientations
    x0: np.ndarray             # [2S, 3] sphere positions
    side: float = 0.0
    seed: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return 2 * self.S

    def phys(self) -> dict:
        return dict(a=self.a, mu=self.mu, k0=self.k0, ell=self.ell, omega=self.omega,
                    lam=self.lam, phi=self.phi)


def side_for_density(S: int, density: float) -> float:
    """Cube side that holds S centres at the given number density."""
    return (S / density) ** (1.0 / 3.0)


def _centres(rng: np.random.Generator, S: int, side: float, min_sep: float) -> np.ndarray:
    """Uniform centres in the cube, rejection by minimum separation (cell grid)."""
    out = np.empty((S, 3))
    if min_sep <= 0:
        return rng.uniform(-side / 2, side / 2, size=(S, 3))
    cell = min_sep
    ncell = max(1, int(math.floor(side / cell)))
    grid: dict = {}
    n = 0
    tries = 0
    while n < S:
        tries += 1
        if tries > 1000 * S + 10000:
            raise RuntimeError("could not place centres: cube too small for min_sep")
        p = rng.uniform(-side / 2, side / 2, size=3)
        c = tuple(np.minimum(((p + side / 2) / cell).astype(int), ncell - 1))
        ok = True
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    for j in grid.get((c[0] + dx, c[1] + dy, c[2] + dz), ()):
                        if np.sum((out[j] - p) ** 2) < min_sep * min_sep:
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if not ok:
                break
        if ok:
            out[n] = p
            grid.setdefault(c, []).append(n)
            n += 1
    return out


def _orientations(rng: np.random.Generator, S: int) -> np.ndarray:
    z = rng.uniform(-1.0, 1.0, size=S)
    az = rng.uniform(0.0, 2.0 * math.pi, size=S)
    rxy = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([rxy * np.cos(az), rxy * np.sin(az), z], axis=1)


def spheres_at_rest(R: np.ndarray, N: np.ndarray, ell: float, lam: np.ndarray,
                    phi: np.ndarray) -> np.ndarray:
    """Sphere positions R -/+ N L(0)/2 with L(0) = ell + lam sin(phi) (Sec. IV start)."""
    L0 = ell + lam * np.sin(phi)
    x = np.empty((2 * R.shape[0], 3))
    x[0::2] = R - 0.5 * L0[:, None] * N
    x[1::2] = R + 0.5 * L0[:, None] * N
    return x


def make_suspension(S: int, *, seed: int = 0, side: float | None = None, density: float = 0.002,
                    min_sep: float = 2.0, a: float = 0.05, mu: float = 1.0, k0: float = 1.0,
                    ell: float = 1.0, period: float = 1.0, lam: float | np.ndarray = 0.2,
                    dt: float = 1e-3, mobility: str = "rpy",
                    phases: np.ndarray | None = None) -> Suspension:
    """Random suspension with the parameters of the paper-scale workloads."""
    if side is None:
        side = side_for_density(S, density)
    rng = np.random.default_rng(seed)
    R = _centres(rng, S, side, min_sep)
    Nv = _orientations(rng, S)
    phi = rng.uniform(0.0, 2.0 * math.pi, size=S) if phases is None else np.asarray(phases, float)
    lam_arr = np.full(S, float(lam)) if np.isscalar(lam) else np.asarray(lam, float).copy()
    x0 = spheres_at_rest(R, Nv, ell, lam_arr, phi)
    return Suspension(S=S, a=a, mu=mu, k0=k0, ell=ell, omega=2 * math.pi / period, dt=dt,
                      mobility=mobility, lam=lam_arr, phi=phi, R0=R, N0=Nv, x0=x0, side=side,
                      seed=seed)


# ---------------------------------------------------------------------------
# Named workloads (sizes as the benchmarks and parity tests use them)
# ---------------------------------------------------------------------------

def small_fp64_oseen(seed: int = 0) -> Suspension:
    """S=16 (N=32), cube side 8, min separation 2, Oseen, dt=1e-3, lambda=0.2."""
    return make_suspension(16, seed=seed, side=8.0, mobility="oseen")


def paper_scale(S: int = 512, seed: int = 0, mobility: str = "rpy") -> Suspension:
    """S dumbbells at number density 0.002 (S=512: N=1024, side 63.5), lambda=0.2."""
    return make_suspension(S, seed=seed, density=0.002, mobility=mobility)


def ensemble_sizes(count: int = 256, lo: int = 8, hi: int = 2048, seed: int = 0) -> np.ndarray:
    """Dumbbell counts log-uniform in [lo, hi] (rounded), one per system."""
    rng = np.random.default_rng(seed)
    return np.round(np.exp(rng.uniform(math.log(lo), math.log(hi), size=count))).astype(int)


def ensemble(count: int = 256, lo: int = 8, hi: int = 2048, seed0: int = 0,
             mobility: str = "rpy") -> list[Suspension]:
    """Independent systems: S log-uniform in [lo, hi], lambda ~ U[0.1, 0.3] per system,
    system k drawn from seed seed0 + k at density 0.002."""
    sizes = ensemble_sizes(count, lo, hi, seed=seed0)
    out = []
    for k, S in enumerate(sizes):
        lam = float(np.random.default_rng(10_000 + seed0 + k).uniform(0.1, 0.3))
        out.append(make_suspension(int(S), seed=seed0 + k, lam=lam, mobility=mobility))
    return out


def request_trace(n: int = 500, rate: float = 200.0, sizes=(16, 64, 256, 1024, 4096),
                  steps_lo: float = 1e3, steps_hi: float = 1e5, seed: int = 0):
    """Poisson arrivals (mean ``rate``/s): (arrival_s, S, steps, seed) per request."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=n)
    arr = np.cumsum(gaps)
    S = rng.choice(np.asarray(sizes), size=n)
    steps = np.round(np.exp(rng.uniform(math.log(steps_lo), math.log(steps_hi), size=n))).astype(int)
    return [(float(arr[i]), int(S[i]), int(steps[i]), int(i)) for i in range(n)]


# ---------------------------------------------------------------------------
# Workloads of the paper's other experiments
# ---------------------------------------------------------------------------

def colloids(N: int, *, seed: int = 0, density: float = 0.002, min_sep: float = 2.0, a: float = 0.05,
             mu: float = 1.0, force=(0.0, 0.0, -1.0), dt: float = 1e-3,
             mobility: str = "oseen") -> tuple[Suspension, np.ndarray]:
    """N colloidal spheres under one constant force (Sec. IV speed-up test: colloids
    moving under a constant applied force, Oseen interactions).  Spheres are
    paired as spring-less dumbbells (k0 = 0, lambda = 0) so the dumbbell
    machinery carries them; returns the suspension and the force [N, 3]."""
    if N % 2:
        raise ValueError("N must be even")
    S = N // 2
    side = (N / density) ** (1.0 / 3.0)
    rng = np.random.default_rng(seed)
    x = _centres(rng, N, side, min_sep)
    s = Suspension(S=S, a=a, mu=mu, k0=0.0, ell=1.0, omega=2 * math.pi, dt=dt, mobility=mobility,
                   lam=np.zeros(S), phi=np.zeros(S), R0=0.5 * (x[0::2] + x[1::2]),
                   N0=np.tile([1.0, 0.0, 0.0], (S, 1)), x0=x, side=side, seed=seed)
    F = np.tile(np.asarray(force, float), (N, 1))
    return s, F


def lattice(x: int, spacing: float, *, seed: int = 0, phases: str = "checkerboard",
            ell: float = 5e-6, a_over_ell: float = 0.2, lam_over_ell: float = 0.1,
            omega: float = 500.0, k0: float = 1e-3, mu: float = 1e-3, dt_over_T: float = 1e-4,
            mobility: str = "rpy") -> Suspension:
    """Dumbbell centres on an x*x*x cubic lattice of the given spacing (Sec. III.C),
    orientations uniform on the sphere (seeded), phases either the 3d
    checkerboard {0, pi/2} (alternating between nearest neighbours) or uniform
    on [0, 2pi).  Default parameters are those of Fig. 1 (SI units)."""
    rng = np.random.default_rng(seed)
    idx = np.stack(np.meshgrid(np.arange(x), np.arange(x), np.arange(x), indexing="ij"), -1).reshape(-1, 3)
    R = (idx - (x - 1) / 2.0) * spacing
    S = R.shape[0]
    Nv = _orientations(rng, S)
    if phases == "checkerboard":
        phi = np.where(idx.sum(1) % 2 == 0, 0.0, math.pi / 2)
    elif phases == "random":
        phi = rng.uniform(0.0, 2 * math.pi, size=S)
    else:
        raise ValueError(phases)
    lam = np.full(S, lam_over_ell * ell)
    x0 = spheres_at_rest(R, Nv, ell, lam, phi)
    T = 2 * math.pi / omega
    return Suspension(S=S, a=a_over_ell * ell, mu=mu, k0=k0, ell=ell, omega=omega,
                      dt=dt_over_T * T, mobility=mobility, lam=lam, phi=phi, R0=R, N0=Nv, x0=x0,
                      side=spacing * x, seed=seed, meta={"phases": phases, "spacing": spacing})
