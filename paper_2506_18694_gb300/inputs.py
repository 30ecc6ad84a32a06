"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds no arithmetic of the solver: it only draws random numbers and
samples the analytic source f(x) = a exp(-|x - x0|^2 / (2 sigma^2)) at the grid
nodes (x fastest).  Turning f into a load vector b = M f is the solver's job
(``rhs_kind = nodal`` in the C-ABI) and the oracle's job, each on its own.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

SOMMERFELD = 0
DIRICHLET = 1


@dataclass(frozen=True)
class Workload:
    """One configuration of the solver: grid, wavenumber, shifts, boundary tags, source."""

    name: str
    dim: int
    n: int
    k: float
    delta: float
    delta_hat: float
    bc: tuple
    centre: tuple
    sigma: float = 0.05
    amplitude: complex = 1.0 + 0.0j
    tol: float = 1e-8

    @property
    def nodes(self) -> int:
        return (self.n + 1) ** self.dim


def _uniform_centre(seed, dim):
    rng = np.random.default_rng(seed)
    return tuple(float(v) for v in rng.uniform(0.0, 1.0, size=dim))


def workload(name: str, delta_hat: str | float = "k") -> Workload:
    """The named configurations (2D 32^2 k=10, 2D 512^2 k=80, 3D 128^3 k=40).

    ``delta_hat`` is ``"k"`` (the shift equal to the wavenumber) or a number
    (2.0 is the value used throughout the paper's experiments, Sec. 5.1).
    """
    if name == "2d_n32_k10":
        dim, n, k, bc, c = 2, 32, 10.0, (SOMMERFELD,) * 4, (0.5, 0.5)
    elif name == "2d_n512_k80":
        dim, n, k, bc, c = 2, 512, 80.0, (SOMMERFELD,) * 4, _uniform_centre(2, 2)
    elif name == "3d_n128_k40":
        dim, n, k = 3, 128, 40.0
        bc = (SOMMERFELD,) * 4 + (DIRICHLET, SOMMERFELD)
        c = (0.5, 0.5, 0.5)
    else:
        raise KeyError(name)
    dh = k if delta_hat == "k" else float(delta_hat)
    return Workload(name, dim, n, k, 0.0, dh, bc, c)


def node_coords(dim: int, n: int) -> np.ndarray:
    """(N, dim) float64 coordinates of the nodes of the uniform grid, x fastest."""
    t = np.arange(n + 1) / n
    grids = np.meshgrid(*([t] * dim)[::-1], indexing="ij")[::-1]
    return np.stack([g.ravel() for g in grids], axis=1)


def gaussian_source(dim: int, n: int, centre, sigma: float = 0.05,
                    amplitude: complex = 1.0) -> np.ndarray:
    """Nodal values of a exp(-|x - x0|^2 / (2 sigma^2)) as complex128, x fastest."""
    x = node_coords(dim, n)
    r2 = ((x - np.asarray(centre)[None, :]) ** 2).sum(axis=1)
    return (amplitude * np.exp(-r2 / (2.0 * sigma * sigma))).astype(np.complex128)


def random_complex(N: int, seed: int) -> np.ndarray:
    """Standard complex normal entries (real and imaginary parts N(0,1)), complex128."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(N) + 1j * rng.standard_normal(N)


def batch_sources(count: int = 64, n: int = 256, seed: int = 4):
    """Batched 2D problems: k drawn from {20, 40, 80}, uniform centres, amplitudes g1 + i g2 with g ~ N(0,1)."""
    rng = np.random.default_rng(seed)
    ks = rng.choice(np.array([20.0, 40.0, 80.0]), size=count)
    centres = rng.uniform(0.0, 1.0, size=(count, 2))
    amps = rng.standard_normal(count) + 1j * rng.standard_normal(count)
    return [(float(ks[i]), tuple(centres[i]), complex(amps[i])) for i in range(count)]


@dataclass(frozen=True)
class BatchWorkload:
    """A batch of 2D problems on one grid: per-problem k, source centre and amplitude."""

    name: str
    dim: int
    n: int
    ks: tuple
    centres: tuple
    amplitudes: tuple
    delta: float
    delta_hats: tuple
    bc: tuple
    sigma: float = 0.05
    tol: float = 1e-8

    @property
    def count(self) -> int:
        return len(self.ks)

    @property
    def nodes(self) -> int:
        return (self.n + 1) ** self.dim

    def sources(self) -> np.ndarray:
        """(count, nodes) nodal source values, problem after problem."""
        return np.stack([gaussian_source(self.dim, self.n, c, self.sigma, a)
                         for c, a in zip(self.centres, self.amplitudes)])


def batch_workload(name: str = "2d_batch64_n256", delta_hat: str | float = "k") -> BatchWorkload:
    """64 right sides on the 2D 256^2 grid (Sommerfeld on all sides), k drawn from {20, 40, 80}
    with seed 4, uniform centres, complex normal amplitudes; delta_hat = k or a number."""
    if name != "2d_batch64_n256":
        raise KeyError(name)
    src = batch_sources(64, 256, 4)
    ks = tuple(s[0] for s in src)
    dhs = ks if delta_hat == "k" else tuple(float(delta_hat) for _ in ks)
    return BatchWorkload(name, 2, 256, ks, tuple(s[1] for s in src), tuple(s[2] for s in src), 0.0, dhs,
                         (SOMMERFELD,) * 4)


@dataclass(frozen=True)
class ServeRequest:
    """One request of the serving workload: its grid, wavenumber, source and arrival time."""

    dim: int
    n: int
    k: float
    delta: float
    delta_hat: float
    bc: tuple
    centre: tuple
    amplitude: complex
    arrival: float = 0.0
    sigma: float = 0.05

    @property
    def nodes(self) -> int:
        return (self.n + 1) ** self.dim

    def source(self) -> np.ndarray:
        return gaussian_source(self.dim, self.n, self.centre, self.sigma, self.amplitude)


def serving_requests(count: int = 1000, seed: int = 5, rate: float = 1.0, delta_hat: str | float = "k"):
    """Requests of the serving workload: half 2D with n log-uniform in [64, 1024], half 3D
    with n log-uniform in [32, 96], n rounded to a multiple of 8; k uniform in [10, 160]
    capped at 2 pi n / 10 (at least 10 points per wavelength); Gaussian sources (sigma
    0.05) at uniform centres with complex normal amplitudes; Poisson arrivals at `rate`
    per second.  2D: Sommerfeld on all sides; 3D: u = 0 on z = 0, Sommerfeld elsewhere."""
    rng = np.random.default_rng(seed)
    out, t = [], 0.0
    for _ in range(count):
        dim = 2 if rng.uniform() < 0.5 else 3
        lo, hi = (64, 1024) if dim == 2 else (32, 96)
        n = int(round(np.exp(rng.uniform(np.log(lo), np.log(hi))) / 8.0)) * 8
        n = min(max(n, lo), hi)
        k = float(min(rng.uniform(10.0, 160.0), 2.0 * np.pi * n / 10.0))
        bc = (SOMMERFELD,) * 4 if dim == 2 else (SOMMERFELD,) * 4 + (DIRICHLET, SOMMERFELD)
        centre = tuple(float(v) for v in rng.uniform(0.0, 1.0, size=dim))
        amp = complex(rng.standard_normal(), rng.standard_normal())
        t += rng.exponential(1.0 / rate)
        dh = k if delta_hat == "k" else float(delta_hat)
        out.append(ServeRequest(dim, n, k, 0.0, dh, bc, centre, amp, t))
    return out


def uneven_requests(count: int = 48, seed: int = 6):
    """Solves on uneven 2D grids (the packed-launch workload): n uniform in {64, 96, ..., 256},
    k uniform in {20, 40}, delta = 0, delta_hat = k, Sommerfeld on all sides, Gaussian sources
    at uniform centres with complex normal amplitudes; all arrive at once."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.choice([64, 96, 128, 160, 192, 224, 256]))
        k = float(rng.choice([20.0, 40.0]))
        centre = tuple(float(v) for v in rng.uniform(0.0, 1.0, size=2))
        amp = complex(rng.standard_normal(), rng.standard_normal())
        out.append(ServeRequest(2, n, k, 0.0, k, (SOMMERFELD,) * 4, centre, amp, 0.0))
    return out
