"""PCG (Algorithm 1), step-size search (Algorithm 2) and CM-PCG (Algorithm 3).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The iteration follows Section 3.1 in the paper's order:
  mu_n, r^n = H(Phi^n) - mu_n Phi^n, preconditioned residual, Polak-Ribiere+
  beta^n, D^n, tangent projection P^n (Eq. formula-project), P^n/||P^n||,
  step size theta_n (Algorithm 2 with the quadratic model of Eqs. approeng-bn),
  Phi^{n+1} = cos(theta) Phi^n + sin(theta) P^n/||P^n|| (Eq. formula-pcg),
  then the stopping test (Section 3.4, Eqs. stop1-stop3).

Readings (written independently on the CUDA side):
  R-STEP   theta_trial = 0.1, sigma = 1/2 ("halve it"), at most 40 halvings;
           if none decreases the energy the iterate is kept and the solve ends
           with status "stagnated".  The halving applies to both branches.
  R-DE     "the energy decreases" means DeltaE(theta) = E(cos(theta) Phi^n +
           sin(theta) P^n/||P^n||) - E(Phi^n) < 0, with DeltaE evaluated from the
           explicit sin/cos form of E(theta) that Section 3.1 describes
           (Model.energy_change): a difference of two O(1) energies cannot
           resolve the O(||r||^2) decrease near the minimiser in FP64.
  R-RESET  Step 2's "set beta = 0 and go to Step 1" recomputes D = -P r, P,
           P/||P||, a_n, b_n once.  If the test still fails with beta = 0
           (possible only through rounding when r ~ 0) the solve ends "stagnated".
  R-PRP    beta uses the stored s_{n-1} = Re<r^{n-1}, P r^{n-1}> (preconditioner
           of step n-1) and the current preconditioner in the numerator;
           beta = 0 at n = 0 and at the start of every multigrid level.
  R-NORM   Phi^{n+1} is renormalised to unit mass after the update (Eq. update).
  R-STOP   the test is evaluated at the start of iteration n (n >= 1) on the
           new iterate: stop3 |DeltaE(theta_{n-1})| < tol (the accepted step's
           energy change, R-DE; equal to E(Phi^n) - E(Phi^{n-1}) up to rounding), stop2
           max_l ||r_l^n||_inf < tol, stop1 max_l ||phi_l^n - phi_l^{n-1}||_inf
           < tol.  `res_tol`, if set, additionally requires ||r^n||_inf < res_tol.
  R-EXACT  line_search="exact" solves Eq. theta instead of the quadratic model (see
           exact_theta); Algorithm 2's acceptance test and halvings still apply.
  R-CM     interpolation between levels is spectral zero padding: coefficient
           p in [-N/2, N/2-1] is placed at the same p on the 2N grid, the result
           is scaled by 2^d and renormalised to unit mass; each level restarts
           PCG (beta = 0) with the same stopping rule.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .fft import fftn, ifftn
from .model import Grid, Model


@dataclass
class Options:
    stop: str = "energy"          # "energy" (Eq. stop3), "residual" (Eq. stop2), "dphi" (Eq. stop1)
    tol: float = 1e-12
    res_tol: float | None = None  # extra residual requirement (parity runs)
    max_iter: int = 20000
    theta_trial: float = 0.1
    sigma: float = 0.5
    max_halvings: int = 40
    precond: str = "combined"     # "combined" (Eq. PreCondMix), "kinetic", "potential", "none"
    line_search: str = "model"    # "model": Algorithm 2's quadratic model; "exact": Eq. theta (R-EXACT)


@dataclass
class Result:
    Phi: np.ndarray
    energy: float
    mu: float
    masses: list
    iters: int
    status: str                     # "converged", "max_iter", "stagnated"
    res_inf: float
    energies: list = field(default_factory=list)
    dE_last: float | None = None
    beta_resets: int = 0
    halvings: int = 0


def _apply_precond(model: Model, kind: str, r, Phi, alpha):
    if kind == "combined":
        return model.precond_C(r, Phi, alpha)
    if kind == "kinetic":
        return model.precond_kin(r, Phi, alpha)
    if kind == "potential":
        return model.precond_pot(r, Phi, alpha)
    if kind == "none":
        return r.copy()
    raise ValueError(kind)


def exact_theta(model: Model, Phi, Phat, t0: float) -> float:
    """theta_n = argmin_{theta > 0} E(cos(theta) Phi + sin(theta) Phat) (Eq. theta), on the
    explicit sin/cos form of E(theta) (Section 3.1).  R-EXACT: E(theta) has period pi (the
    energy does not see the sign of the wave function) and decreases at 0+; the minimiser
    taken is the first zero of dE/dtheta found by doubling from the quadratic model's theta
    t0 (a bracket [lo, hi] with dE/dtheta(lo) < 0 <= dE/dtheta(hi), hi <= pi), solved to
    rounding by Brent's root finder.  If no sign change is met up to pi, t0 is kept."""
    from scipy.optimize import brentq
    _, g = model.trig_form(Phi, Phat)
    lo, hi = 0.0, min(t0, math.pi)
    while g(hi) < 0.0 and hi < math.pi:
        lo, hi = hi, min(2.0 * hi, math.pi)
    if g(hi) < 0.0:
        return t0
    return brentq(g, lo, hi, xtol=1e-300, rtol=4 * np.finfo(float).eps, maxiter=500)


def normalize(model: Model, Phi):
    return Phi / math.sqrt(model.mass(Phi))


def pcg(model: Model, Phi0, opts: Options = Options(), callback=None) -> Result:
    """Algorithm 1 with Algorithm 2 (Section 3.1)."""
    Phi = normalize(model, np.array(Phi0, dtype=np.complex128))
    E = model.energy(Phi)
    energies = [E]
    r_prev = P_prev = None
    s_prev = None
    Phi_prev = None
    dE_last = None
    resets = halvings = 0
    n = 0
    status = "max_iter"
    while True:
        HPhi = model.H(Phi)
        mu = model.mu(Phi, HPhi)
        r = HPhi - mu * Phi
        res_inf = float(np.max(np.abs(r)))
        # stopping test on the current iterate (R-STOP)
        if n >= 1 or opts.stop == "residual":
            if opts.stop == "energy":
                ok = abs(dE_last) < opts.tol
            elif opts.stop == "residual":
                ok = res_inf < opts.tol
            elif opts.stop == "dphi":
                ok = float(np.max(np.abs(Phi - Phi_prev))) < opts.tol
            else:
                raise ValueError(opts.stop)
            if ok and opts.res_tol is not None:
                ok = res_inf < opts.res_tol
            if ok:
                status = "converged"
                break
        if n >= opts.max_iter:
            break
        alpha = model.alpha(Phi)
        Pr = _apply_precond(model, opts.precond, r, Phi, alpha)
        s_cur = model.inner(r, Pr).real
        if n == 0 or P_prev is None:
            beta = 0.0
        else:
            beta = max(model.inner(r - r_prev, Pr).real / s_prev, 0.0)
        # Algorithm 2, Steps 1-2 (R-RESET)
        while True:
            D = -Pr + beta * P_prev if beta != 0.0 else -Pr
            P = D - model.inner(D, Phi).real * Phi
            a, b = model.step_coefficients(Phi, P, HPhi, mu)
            if b > 0 or (b == 0 and a >= 0):
                if beta == 0.0:
                    status = "stagnated"
                    break
                beta = 0.0
                resets += 1
                continue
            theta = -b / (2.0 * a) if (a > 0 and b < 0) else opts.theta_trial
            break
        if status == "stagnated":
            break
        Phat = P / math.sqrt(model.mass(P))
        if opts.line_search == "exact":
            theta = exact_theta(model, Phi, Phat, theta)
        # Algorithm 2, Steps 3-4
        accepted = False
        for _ in range(opts.max_halvings + 1):
            dE = model.energy_change(Phi, Phat, theta)
            if dE < 0:
                accepted = True
                break
            theta *= opts.sigma
            halvings += 1
        if not accepted:
            status = "stagnated"
            break
        Phi_prev = Phi
        Phi = normalize(model, math.cos(theta) * Phi + math.sin(theta) * Phat)
        r_prev, P_prev, s_prev = r, P, s_cur
        dE_last = dE
        E = model.energy(Phi)
        energies.append(E)
        n += 1
        if callback is not None:
            callback(n, Phi, E)
    HPhi = model.H(Phi)
    mu = model.mu(Phi, HPhi)
    res_inf = float(np.max(np.abs(HPhi - mu * Phi)))
    return Result(Phi=Phi, energy=E, mu=mu, masses=model.masses(Phi), iters=n, status=status,
                  res_inf=res_inf, energies=energies, beta_resets=resets, halvings=halvings,
                  dE_last=dE_last)


def prolong(Phi, coarse: Grid, fine: Grid):
    """R-CM: spectral zero padding from `coarse` to `fine` (sizes doubled on every axis)."""
    d = coarse.d
    Ph = fftn(Phi, coarse.stack_axes)
    out = np.zeros((3,) + fine.shape, dtype=np.complex128)
    idx = []
    for ax in range(d):  # numpy axis order: z, y, x -> physical axis d-1-...
        nc = coarse.n[d - 1 - ax]
        nf = fine.n[d - 1 - ax]
        p = np.arange(nc)
        p = np.where(p < nc // 2, p, p - nc)
        idx.append(np.mod(p, nf))
    out[(slice(None),) + np.ix_(*idx)] = Ph
    fineP = ifftn(out, fine.stack_axes) * (2 ** d)
    return fineP


def cm_pcg(models, Phi0, opts: Options = Options()) -> tuple[Result, list]:
    """Algorithm 3: PCG on each level of `models` (coarse to fine, each grid the
    previous one refined by 2 on every axis), prolongation between levels."""
    results = []
    Phi = Phi0
    for lev, m in enumerate(models):
        if lev > 0:
            Phi = prolong(results[-1].Phi, models[lev - 1].grid, m.grid)
            Phi = normalize(m, Phi)
        res = pcg(m, Phi, opts)
        results.append(res)
    return results[-1], results
