"""Shared helpers of the GPU parity tests (oracle models for given problems)."""
import numpy as np

from oracle.model import Grid, Model, Trap


def oracle_model(n, L, par, trap=None):
    trap = trap or {}
    kind = trap.get("kind", 0)
    g = tuple(trap.get("g", (1.0, 1.0, 1.0)))
    quad = trap.get("quad", 0.0) if kind else 0.0
    quart = trap.get("quart", 0.0) if kind else 0.0
    user = trap.get("user_V") if kind == 2 else None
    return Model(Grid(n, L), Trap(g=g, quad=quad, quart=quart, user=user), Omega=par[0], gamma=par[1],
                 c0=par[2], c1=par[3])


def rel_max(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))
