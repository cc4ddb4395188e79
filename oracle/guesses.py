"""Initial guesses (a)-(f) of Section 4 (oracle; test infrastructure only).

phi_a = pi^{-d/4} exp(-|x|^2/2); phi_b = (x + i y) phi_a; bar = complex conjugate;
c = (a + b)/||a + b||; d = ((1-Omega) a + Omega b)/||.||; e = (Omega a + (1-Omega) b)/||.||;
f = phi_TF/||phi_TF|| with the Thomas-Fermi profile sqrt((mu_TF - V)/c0)_+ and
mu_TF = 1/2 (4 c0 gx gy / pi)^{1/2} (2D), 1/2 (15 c0 gx gy gz / (4 pi))^{2/5} (3D).
Norms are the discrete L2 norms on the grid.  A spin-1 guess is
(phi_1, phi_0, phi_-1)/sqrt(3) (Section 4, the 10^3 combinations).
Kinds: 0=a 1=b 2=b_bar 3=c 4=c_bar 5=d 6=d_bar 7=e 8=e_bar 9=f.
"""
from __future__ import annotations

import math

import numpy as np

from .model import Model

KINDS = ["a", "b", "b_bar", "c", "c_bar", "d", "d_bar", "e", "e_bar", "f"]


def single(model: Model, kind: int) -> np.ndarray:
    g = model.grid
    r2 = sum(x * x for x in g.X)
    pa = math.pi ** (-g.d / 4.0) * np.exp(-r2 / 2.0)
    pb = (g.X[0] + 1j * g.X[1]) * pa
    nrm = lambda f: f / math.sqrt(g.integrate(np.abs(f) ** 2))
    W = model.Omega
    name = KINDS[kind]
    if name == "a":
        return pa.astype(np.complex128)
    if name == "b":
        return pb
    if name == "b_bar":
        return np.conj(pb)
    if name in ("c", "c_bar"):
        f = nrm(pa + pb)
    elif name in ("d", "d_bar"):
        f = nrm((1 - W) * pa + W * pb)
    elif name in ("e", "e_bar"):
        f = nrm(W * pa + (1 - W) * pb)
    elif name == "f":
        if model.c0 <= 0:
            raise ValueError("guess (f) needs c0 > 0")
        gx, gy = model.trap.g[0], model.trap.g[1]
        if g.d == 2:
            muTF = 0.5 * math.sqrt(4.0 * model.c0 * gx * gy / math.pi)
        else:
            gz = model.trap.g[2]
            muTF = 0.5 * (15.0 * model.c0 * gx * gy * gz / (4.0 * math.pi)) ** 0.4
        tf = np.sqrt(np.maximum(muTF - model.V, 0.0) / model.c0)
        return nrm(tf).astype(np.complex128)
    else:
        raise ValueError(kind)
    return np.conj(f) if name.endswith("_bar") else f


def spin1(model: Model, kinds) -> np.ndarray:
    """(phi_1, phi_0, phi_-1)/sqrt(3) with each component of the given kind."""
    return np.stack([single(model, k) for k in kinds]) / math.sqrt(3.0)
