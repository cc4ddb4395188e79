"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and bench.py.

This module holds no arithmetic of the method (no operators, energies or
iteration steps): it only draws pseudo-random numbers and lays initial wave
functions and physical parameters out on a grid.  Both the CPU oracle and the
CUDA path receive the exact same host arrays from here.

Random numbers: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), uniform doubles from the top 53 bits.

Layout of a wave function: complex128 array of shape (3, Ny, Nx) in 2D or
(3, Nz, Ny, Nx) in 3D; component order (phi_1, phi_0, phi_-1); x fastest.
Grid points x_m = -L + m h, h = 2L/N, m = 0..N-1 (Section 3.2 of the paper).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_MASK = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 stream; `next()` returns a Python int in [0, 2^64)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next() >> 11) * (1.0 / 9007199254740992.0)

    def uniform_in(self, lo: float, hi: float) -> float:
        return lo + (hi - lo) * self.uniform()

    def randint(self, lo: int, hi: int) -> int:
        """Integer uniform in [lo, hi] inclusive."""
        return lo + int(self.uniform() * (hi - lo + 1))


def seed_for(config: int, solve_index: int) -> int:
    """Seed of solve `solve_index` of workload `config` (1000*config + index)."""
    return 1000 * config + solve_index


def axes(n, L):
    """Per-axis coordinate vectors (x, y[, z]) for grid sizes n and half-widths L."""
    return [(-Lk + np.arange(nk) * (2.0 * Lk / nk)) for nk, Lk in zip(n, L)]


def mesh(n, L):
    """Coordinate arrays X, Y[, Z] shaped like one component (z, y, x order)."""
    ax = axes(n, L)
    grids = np.meshgrid(*ax[::-1], indexing="ij")  # slowest axis first
    return grids[::-1]  # return in (X, Y[, Z]) order


def _mass(phi, n, L):
    h = np.prod([2.0 * Lk / nk for nk, Lk in zip(n, L)])
    return h * float(np.sum(np.abs(phi) ** 2))


def gaussian_guess(n, L, seed: int, vortex: bool = False) -> np.ndarray:
    """Seeded Gaussian (optionally times a vortex phase) initial guess.

    Per component: exp(-sum_i (x_i - c_i)^2 / (2 w^2)) * exp(i t) with
    c_i ~ U[-1,1], w ~ U[0.8,1.2], t ~ U[0, 2 pi); the vortex form multiplies
    by prod_j ((x - a_j) + i (y - b_j)), m ~ U{1,2,3}, (a_j, b_j) ~ U[-1.5,1.5]^2.
    Each component is scaled to mass 1/3 so the total mass is 1.
    """
    rng = SplitMix64(seed)
    X = mesh(n, L)
    d = len(n)
    out = np.empty((3,) + X[0].shape, dtype=np.complex128)
    for comp in range(3):
        c = [rng.uniform_in(-1.0, 1.0) for _ in range(d)]
        w = rng.uniform_in(0.8, 1.2)
        t = rng.uniform_in(0.0, 2.0 * math.pi)
        r2 = sum((X[i] - c[i]) ** 2 for i in range(d))
        phi = np.exp(-r2 / (2.0 * w * w)) * complex(math.cos(t), math.sin(t))
        if vortex:
            m = rng.randint(1, 3)
            for _ in range(m):
                a = rng.uniform_in(-1.5, 1.5)
                b = rng.uniform_in(-1.5, 1.5)
                phi = phi * ((X[0] - a) + 1j * (X[1] - b))
        phi = phi / math.sqrt(3.0 * _mass(phi, n, L))
        out[comp] = phi
    return out


@dataclass
class Params:
    Omega: float
    gamma: float
    beta0: float
    beta1: float


def batch_params(seed: int, count: int) -> list[Params]:
    """Parameter draws of the batched sweep: Omega~U[0,0.95], gamma~U[0,2],
    beta0~U[100,2000], beta1~U[-10,10] (one SplitMix64 stream)."""
    rng = SplitMix64(seed)
    out = []
    for _ in range(count):
        out.append(Params(rng.uniform_in(0.0, 0.95), rng.uniform_in(0.0, 2.0),
                          rng.uniform_in(100.0, 2000.0), rng.uniform_in(-10.0, 10.0)))
    return out


def random_state(n, seed: int) -> np.ndarray:
    """Unstructured complex field (3, *shape) with entries ~ U[-1,1] + i U[-1,1].

    Used for operator-level tests (the whole spectrum is excited)."""
    rng = np.random.default_rng(seed)
    shape = (3,) + tuple(n[::-1])
    return rng.uniform(-1, 1, shape) + 1j * rng.uniform(-1, 1, shape)


def smooth_random_state(n, L, seed: int, width: float = 1.5) -> np.ndarray:
    """Random smooth, localised complex field: a random field damped by a
    Gaussian envelope of the given width (decays to ~0 at the box edge)."""
    X = mesh(n, L)
    env = np.exp(-sum(x * x for x in X) / (2 * width * width))
    return random_state(n, seed) * env[None]


# grids of the served trace: (n, L) with their draw weights
SERVE_GRIDS = [((64, 64), (12.0, 12.0)), ((128, 128), (12.0, 12.0)), ((256, 256), (12.0, 12.0)),
               ((512, 512), (12.0, 12.0)), ((64, 64, 64), (8.0, 8.0, 8.0)), ((128, 128, 128), (8.0, 8.0, 8.0))]
SERVE_WEIGHTS = [0.30, 0.25, 0.20, 0.10, 0.10, 0.05]


def serve_trace(seed: int, count: int, rate: float):
    """Served-trace requests: Poisson arrivals at `rate` per second (exponential
    gaps), a grid drawn from SERVE_GRIDS by SERVE_WEIGHTS, parameters drawn as in
    batch_params, and a guess seed.  Returns dicts sorted by arrival time."""
    rng = SplitMix64(seed)
    pars = batch_params(seed + 1, count)
    cum = np.cumsum(SERVE_WEIGHTS)
    t = 0.0
    out = []
    for k in range(count):
        t += -math.log(1.0 - rng.uniform()) / rate
        g = int(np.searchsorted(cum, rng.uniform() * cum[-1], side="right"))
        g = min(g, len(SERVE_GRIDS) - 1)
        n, L = SERVE_GRIDS[g]
        out.append({"arrival": t, "n": n, "L": L, "params": pars[k], "guess_seed": seed_for(5, k),
                    "vortex": bool(k % 2)})
    return out
