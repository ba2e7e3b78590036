"""Seeded synthetic workloads: sizes, constants and random draws only.

This module is the one place both the CUDA path and the CPU oracle take their
inputs from.  It holds none of the method's arithmetic: no metric, no orbit
formula, no integration.  Random numbers that the method itself draws while it
runs (the rejection sampler of generic bound orbits) are produced on each side
by the SplitMix64 counter-based generator from a seed given here.

Workloads (the paper measures on unspecified random Kerr geodesics, Sec. 6.4;
these synthetic sets stand in for them):
  circular   Schwarzschild, 1024 timelike equatorial circular orbits, radii
             uniform in [6.5M, 20M], dtau = 0.01, 10^4 steps (Sec. 4 orbits).
  camera     Kerr a = 0.9 backward null-ray camera, 1024 x 1024 pixels,
             observer r = 1000M, inclination 80 deg, alpha, beta in [-25M, 25M],
             step 0.05 r, cap 2x10^4, stop at 1.01 r_+ or r > 1100M.
  bound      2^20 generic bound Kerr timelike orbits, spin uniform in
             [0, 0.998]M, periapsis in [ISCO + 0.5M, 10M], eccentricity
             U[0, 0.7], inclination U[0, pi], dtau = 0.02, 10^5 steps.
  bundles    4096 bundles of log-uniform size 64..65536, each with its own
             spin, kind (null camera strip or timelike ensemble) and step cap
             log-uniform in [10^3, 10^5].
  serving    Poisson arrivals mixing camera renders and orbit ensembles.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 1803083200


@dataclass(frozen=True)
class Termination:
    eps_hor: float = 0.01
    r_esc: float = 1100.0
    n_steps_cap: int = 10_000
    dl: float = 0.01
    dl_r_scale: float = 0.0


@dataclass(frozen=True)
class CircularWorkload:
    n: int
    M: float
    a: float
    radii: np.ndarray = field(repr=False)
    term: Termination = Termination()


def circular(n: int = 1024, n_steps: int = 10_000, dtau: float = 0.01, seed: int = SEED_BASE + 1,
             r_lo: float = 6.5, r_hi: float = 20.0) -> CircularWorkload:
    """Schwarzschild circular-orbit ensemble: radii uniform in [r_lo, r_hi] M."""
    rng = np.random.default_rng(seed)
    radii = rng.uniform(r_lo, r_hi, size=n)
    return CircularWorkload(n=n, M=1.0, a=0.0, radii=radii,
                            term=Termination(eps_hor=0.01, r_esc=1100.0, n_steps_cap=n_steps, dl=dtau))


@dataclass(frozen=True)
class CameraWorkload:
    M: float = 1.0
    a: float = 0.9
    r_obs: float = 1000.0
    incl: float = math.radians(80.0)
    fov_half: float = 25.0
    nx: int = 1024
    ny: int = 1024
    term: Termination = Termination(eps_hor=0.01, r_esc=1100.0, n_steps_cap=20_000, dl=0.0,
                                    dl_r_scale=0.05)

    @property
    def n(self) -> int:
        return self.nx * self.ny


def camera(nx: int = 1024, ny: int = 1024, a: float = 0.9, incl_deg: float = 80.0,
           cap: int = 20_000) -> CameraWorkload:
    return CameraWorkload(a=a, incl=math.radians(incl_deg), nx=nx, ny=ny,
                          term=Termination(eps_hor=0.01, r_esc=1100.0, n_steps_cap=cap, dl=0.0,
                                           dl_r_scale=0.05))


@dataclass(frozen=True)
class BoundWorkload:
    n: int
    M: float
    a_max: float
    seed: int
    term: Termination

    def subsample(self, k: int = 1024) -> np.ndarray:
        """Fixed oracle subsample: indices i * (n // k)."""
        step = max(1, self.n // k)
        return np.arange(0, self.n, step, dtype=np.uint64)[:k]


def bound(n: int = 1 << 20, n_steps: int = 100_000, dtau: float = 0.02,
          seed: int = SEED_BASE + 3) -> BoundWorkload:
    return BoundWorkload(n=n, M=1.0, a_max=0.998, seed=seed,
                         term=Termination(eps_hor=0.01, r_esc=1100.0, n_steps_cap=n_steps, dl=dtau))


@dataclass(frozen=True)
class Bundle:
    kind: str          # "camera" (null) or "bound" (timelike)
    n: int             # rays / particles
    a: float           # spin
    cap: int           # step cap
    incl: float        # camera inclination (radians), unused for "bound"
    seed: int          # SplitMix64 seed for "bound"


def bundles(count: int = 4096, seed: int = SEED_BASE + 4, size_lo: int = 64, size_hi: int = 65536,
            cap_lo: float = 1e3, cap_hi: float = 1e5) -> list[Bundle]:
    """Uneven bundles: log-uniform sizes and caps, 50/50 null camera strips and
    timelike bound-orbit ensembles, spin uniform in [0, 0.998]."""
    rng = np.random.default_rng(seed)
    sizes = np.floor(np.exp(rng.uniform(math.log(size_lo), math.log(size_hi), count))).astype(np.int64)
    caps = np.floor(np.exp(rng.uniform(math.log(cap_lo), math.log(cap_hi), count))).astype(np.int64)
    spins = rng.uniform(0.0, 0.998, count)
    kinds = rng.uniform(0.0, 1.0, count) < 0.5
    incl = np.radians(rng.uniform(5.0, 85.0, count))
    seeds = rng.integers(0, 2**62, count)
    return [Bundle("camera" if kinds[i] else "bound", int(sizes[i]), float(spins[i]), int(caps[i]),
                   float(incl[i]), int(seeds[i])) for i in range(count)]


@dataclass(frozen=True)
class Request:
    t_arrival: float
    kind: str
    n: int           # pixels (side^2) or particles
    side: int        # camera side, 0 for ensembles
    a: float
    incl: float
    cap: int
    seed: int


def serving(rate: float, duration: float, seed: int = SEED_BASE + 5, max_side_log2: int = 10,
            max_particles: int = 1 << 18) -> list[Request]:
    """Poisson arrival stream at `rate` req/s for `duration` s: 50% camera renders
    (side 2^U{6..max_side_log2}, a ~ U[0, 0.998], incl ~ U[5, 85] deg, cap 2x10^4),
    50% orbit ensembles (n log-uniform 256..max_particles, cap log-uniform 10^3..10^5)."""
    rng = np.random.default_rng(seed + int(rate))
    t = 0.0
    out: list[Request] = []
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration:
            break
        a = float(rng.uniform(0.0, 0.998))
        if rng.uniform() < 0.5:
            side = 1 << int(rng.integers(6, max_side_log2 + 1))
            out.append(Request(t, "camera", side * side, side, a,
                               math.radians(float(rng.uniform(5.0, 85.0))), 20_000, 0))
        else:
            n = int(math.exp(rng.uniform(math.log(256), math.log(max_particles))))
            cap = int(math.exp(rng.uniform(math.log(1e3), math.log(1e5))))
            out.append(Request(t, "bound", n, 0, a, 0.0, cap, int(rng.integers(0, 2**62))))
    return out
