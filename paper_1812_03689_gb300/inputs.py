"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests
and the benchmark.

This module holds random sampling only -- none of the method's arithmetic --
so that both sides consume identical particle sets.  All workloads live in
the unit cube with equal charges q = 1 / P (total charge 1, eps0 = 1); the
paper's physical units (0.1 fC macro particles, Sec. 6.3) are a linear
rescale that leaves relative errors unchanged.

Gaussian bunches stand in for the paper's multi-bunch cyclotron workloads
(Sec. 6.3, Sec. 7 and the scaling study of Sec. 8): no public dataset is
involved.  Samples outside ``[h0, 1 - h0]^3`` (h0 = base cell width) are
rejected and redrawn, so every cloud-in-cell weight lands inside level 0.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 1812036890


def rng(config_index: int, request_index: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + int(config_index) + 7919 * int(request_index)))


def gaussian_bunches(g: np.random.Generator, n_per_bunch: int, centres, sigma, h0: float,
                     total_charge: float = 1.0):
    """Particles of several Gaussian bunches (one normal per axis), SoA
    float64 ``(x, y, z, q)`` with equal charges summing to total_charge."""
    centres = np.atleast_2d(np.asarray(centres, dtype=np.float64))
    sigma = np.broadcast_to(np.asarray(sigma, dtype=np.float64), (3,))
    parts = []
    for c in centres:
        need = n_per_bunch
        got = []
        while need > 0:
            s = g.normal(size=(int(need * 1.05) + 16, 3)) * sigma + c
            ok = np.all((s >= h0) & (s <= 1.0 - h0), axis=1)
            s = s[ok][:need]
            got.append(s)
            need -= len(s)
        parts.append(np.concatenate(got))
    p = np.concatenate(parts)
    n = len(p)
    q = np.full(n, total_charge / n)
    return (np.ascontiguousarray(p[:, 0]), np.ascontiguousarray(p[:, 1]),
            np.ascontiguousarray(p[:, 2]), q)


def uniform_sphere(g: np.random.Generator, n: int, centre, radius: float, total_charge: float = 1.0):
    """Particles uniformly inside a sphere (the paper's Sec. 6.2 mini-app)."""
    out = []
    need = n
    while need > 0:
        s = g.uniform(-1.0, 1.0, size=(2 * need + 16, 3))
        s = s[np.sum(s * s, axis=1) <= 1.0][:need]
        out.append(s)
        need -= len(s)
    p = np.concatenate(out) * radius + np.asarray(centre)
    q = np.full(n, total_charge / n)
    return (np.ascontiguousarray(p[:, 0]), np.ascontiguousarray(p[:, 1]),
            np.ascontiguousarray(p[:, 2]), q)


@dataclass
class Workload:
    name: str
    n0: int
    lmax: int
    n_particles: int
    centres: list
    sigma: tuple
    tag_mode: str = "rel"
    tag_lambda: float = 0.1
    boxes: list = field(default_factory=list)
    config_index: int = 0

    def particles(self, request_index: int = 0, scale: float = 1.0):
        nb = len(self.centres)
        per = max(1, int(round(self.n_particles * scale / nb)))
        return gaussian_bunches(rng(self.config_index, request_index), per, self.centres, self.sigma,
                                1.0 / self.n0)


def workload(name: str) -> Workload:
    """The named synthetic workloads.

    c1_small: base 32^3, one level (ratio 2) on the central 16^3 coarse cells,
              1e4 particles, isotropic Gaussian sigma 0.08.
    c2_fp64:  base 64^3, two levels tagged at rho > 0.1 max, 1e6 particles,
              anisotropic Gaussian sigmas (0.05, 0.08, 0.12).
    c3_bunches: base 128^3, three levels in total, five bunches (sigma 0.04,
              2e6 each) 0.15 apart along x.
    roofline: base 256^3, three refinement levels, 1e7 particles in the
              five-bunch layout.
    """
    if name == "c1_small":
        return Workload(name, 32, 1, 10_000, [[0.5, 0.5, 0.5]], (0.08, 0.08, 0.08), tag_mode="boxes",
                        boxes=[(1, (16, 16, 16), (47, 47, 47))], config_index=0)
    if name == "c2_fp64":
        return Workload(name, 64, 2, 1_000_000, [[0.5, 0.5, 0.5]], (0.05, 0.08, 0.12), config_index=1)
    five = [[0.2 + 0.15 * i, 0.5, 0.5] for i in range(5)]
    if name == "c3_bunches":
        return Workload(name, 128, 2, 10_000_000, five, (0.04, 0.04, 0.04), config_index=2)
    if name == "roofline":
        return Workload(name, 256, 3, 10_000_000, five, (0.04, 0.04, 0.04), config_index=5)
    raise KeyError(name)


def poisson_arrivals(g: np.random.Generator, n: int, rate_per_s: float):
    """Arrival times (s) of a Poisson process: cumulative exponential gaps."""
    return np.cumsum(g.exponential(1.0 / rate_per_s, size=n))


def log_uniform_int(g: np.random.Generator, lo: float, hi: float, multiple: int = 1) -> int:
    v = math.exp(g.uniform(math.log(lo), math.log(hi)))
    return int(max(lo, min(hi, multiple * round(v / multiple))))


@dataclass
class Request:
    """One independent solve of the batched and served workloads."""
    index: int
    n0: int
    lmax: int
    n_particles: int
    sigma: float
    arrival_s: float = 0.0

    def particles(self, config_index: int):
        g = rng(config_index, self.index + 1)
        return gaussian_bunches(g, self.n_particles, [[0.5, 0.5, 0.5]], (self.sigma,) * 3, 1.0 / self.n0)


def batched_requests(n: int = 256, config_index: int = 3):
    """The batched workload: base grids uniform in 32^3..96^3 (multiples of
    8), 0-2 refinement levels, 1e4-1e5 particles (log-uniform), isotropic
    Gaussian sigma uniform in 0.03..0.1, centre 0.5."""
    g = rng(config_index)
    out = []
    for i in range(n):
        n0 = int(g.integers(4, 13)) * 8
        lmax = int(g.integers(0, 3))
        npart = log_uniform_int(g, 1e4, 1e5)
        sigma = float(g.uniform(0.03, 0.1))
        out.append(Request(i, n0, lmax, npart, sigma))
    return out


def served_requests(n: int = 10_000, rate_per_s: float = 2000.0, config_index: int = 4, max_n0: int = 256,
                    max_particles: float = 1e7):
    """The served workload: Poisson arrivals, base grids log-uniform in
    32^3..max_n0^3 (multiples of 8), 0-3 refinement levels, 1e4..max
    particles (log-uniform), sigma uniform in 0.03..0.1."""
    g = rng(config_index)
    t = poisson_arrivals(g, n, rate_per_s)
    out = []
    for i in range(n):
        n0 = log_uniform_int(g, 32, max_n0, multiple=8)
        lmax = int(g.integers(0, 4))
        npart = log_uniform_int(g, 1e4, max_particles)
        sigma = float(g.uniform(0.03, 0.1))
        out.append(Request(i, n0, lmax, npart, sigma, float(t[i])))
    return out


def sphere_density(lo, hi, h, centre=(0.5, 0.5, 0.5), radius=0.2, total_charge=1.0, sub=8):
    """Charge density of a uniformly charged sphere (the paper's Sec. 6.2
    test) on the cells [lo, hi] (inclusive index box, spacing h) of a level,
    as an array [k, j, i]: each cell's volume fraction inside the sphere
    (sub^3 sample points per cell) times Q / (4/3 pi R^3)."""
    lo = np.asarray(lo)
    hi = np.asarray(hi)
    n = hi - lo + 1
    off = (np.arange(sub) + 0.5) / sub
    out = np.zeros((int(n[2]), int(n[1]), int(n[0])))
    ax = [((np.arange(lo[d], hi[d] + 1)[:, None] + off[None, :]) * h).ravel() for d in range(3)]
    dx2 = (ax[0] - centre[0]) ** 2
    dy2 = (ax[1] - centre[1]) ** 2
    for kk in range(int(n[2])):
        z = ax[2][kk * sub:(kk + 1) * sub]
        dz2 = (z - centre[2]) ** 2
        inside = (dz2[:, None, None] + dy2[None, :, None] + dx2[None, None, :]) < radius * radius
        frac = inside.reshape(sub, int(n[1]), sub, int(n[0]), sub).mean(axis=(0, 2, 4))
        out[kk] = frac
    return out * total_charge / (4.0 / 3.0 * math.pi * radius ** 3)
