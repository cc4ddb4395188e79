"""Discrete model of the rotating spin-orbit-coupled spin-1 condensate (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Wave functions are complex128 stacks of shape (3, Ny, Nx) [2D] or
(3, Nz, Ny, Nx) [3D]; component index 0, 1, 2 holds phi_1, phi_0, phi_-1.
Physical axis x is the last numpy axis.

Sources in the paper:
  * energy functional, spin vector F, spin-1 matrices, SOC operators L0, L1,
    rotation operator Lz, single-particle H0: Section 1 (Eq. energy, the
    explicit F_x, F_y, F_z, the compact matrix F.f and S).
  * Euler-Lagrange operators H_l and chemical potential: Section 2.2
    (Eqs. eigen1-eigen3, muphi); inner product and phase factor (Eq. phase-factor).
  * energy split E1+E2+E3: Section 2.1.  Virial parts: Theorem (Virial identity).
  * Fourier spectral discretisation: Section 3.2 (grid h = 2L/N, x_m = -L + m h,
    wavenumbers v_p = pi p / L, p in [-N/2, N/2-1]).
  * quadratic step model coefficients a_n, b_n and the conjugate bilinear forms
    F~_alpha: Section 3.1 (Eqs. approeng, an, bn).
  * preconditioners P_Delta, P_V, P_C and the shift alpha: Section 3.4
    (Eqs. PreCondKin, PreCnstAlpha, PreCondPot, PreCondMix).

Readings where the paper is silent or ambiguous (shared with the CUDA path,
written independently on each side):
  R-DFT   forward DFT unnormalised, inverse with 1/N per axis (Section 3.2
          omits the 1/N^d in the reconstruction formula).
  R-NYQ   the Nyquist index p = -N/2 keeps v = -pi N / (2L) in every symbol,
          including the odd (first-derivative) ones.
  R-QUAD  integrals are h^d * sum over the N^d periodic nodes; <v,u> = h^d sum v conj(u).
  R-FROZEN in a_n, "H_l(P^n)" is the Hamiltonian with density and spin density
          frozen at Phi^n, applied linearly to P^n.
  R-SOC3D in 3D, L0 and L1 use d/dx and d/dy only.
  R-ALPHA alpha_l is floored at 1e-12 * max_l' |alpha_l'| (and a tiny absolute
          floor); alpha_l + V + c0 rho is floored at 1e-12 * alpha_l pointwise.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .fft import fftn, ifftn

SQ2 = math.sqrt(2.0)


class Grid:
    """Uniform periodic grid on prod_i [-L_i, L_i] (Section 3.2).

    n = (Nx, Ny[, Nz]) even sizes, L = (Lx, Ly[, Lz]).  Arrays are shaped
    (Nz,) Ny, Nx with x the last axis.
    """

    def __init__(self, n, L):
        self.n = tuple(int(k) for k in n)
        self.L = tuple(float(v) for v in L)
        self.d = len(self.n)
        if self.d not in (2, 3) or len(self.L) != self.d:
            raise ValueError("grid must be 2D or 3D")
        for k in self.n:
            if k < 2 or k % 2:
                raise ValueError("grid sizes must be even (Section 3.2: N in 2Z+)")
        self.h = tuple(2.0 * Lk / nk for nk, Lk in zip(self.n, self.L))
        self.dV = float(np.prod(self.h))
        self.shape = tuple(reversed(self.n))
        self.fft_axes = tuple(range(-1, -self.d - 1, -1))  # x, y[, z] numpy axes of a component
        self.stack_axes = tuple(a for a in self.fft_axes)    # same axes on a (3, ...) stack
        self.X = []   # coordinate arrays x, y[, z], broadcastable to self.shape
        self.K = []   # wavenumber arrays v_x, v_y[, v_z] in FFT index order
        for i, (nk, Lk, hk) in enumerate(zip(self.n, self.L, self.h)):
            shp = [1] * self.d
            shp[self.d - 1 - i] = nk
            m = np.arange(nk)
            self.X.append((-Lk + m * hk).reshape(shp))
            p = np.where(m < nk // 2, m, m - nk)  # R-NYQ: index N/2 -> p = -N/2
            self.K.append((math.pi * p / Lk).reshape(shp))
        self.K2 = sum(k * k for k in self.K)

    def integrate(self, f) -> float:
        """R-QUAD: h^d * sum of f over the grid (real part of the result)."""
        return float(np.real(np.sum(f))) * self.dV


@dataclass
class Trap:
    """V = 1/2 sum_i g_i^2 x_i^2 + quad * r^2 + quart * r^4 (+ user array).

    Harmonic (Eq. harmonic): g = trap frequencies.  Harmonic-plus-quartic
    (Eq. harm-quart): g = 0, quad = -0.2, quart = 0.5 (2D).  r^2 sums over all
    d axes.  `user` (array shaped like one component) is added if given."""
    g: tuple = (1.0, 1.0, 1.0)
    quad: float = 0.0
    quart: float = 0.0
    user: np.ndarray | None = None

    def values(self, grid: Grid) -> np.ndarray:
        V = np.zeros(grid.shape)
        r2 = np.zeros(grid.shape)
        for i in range(grid.d):
            V = V + 0.5 * self.g[i] ** 2 * grid.X[i] ** 2
            r2 = r2 + grid.X[i] ** 2
        V = V + self.quad * r2 + self.quart * r2 * r2
        if self.user is not None:
            V = V + np.asarray(self.user, dtype=np.float64).reshape(grid.shape)
        return V


@dataclass
class Model:
    """Grid + trap + physical parameters Omega, gamma, c0 (beta0), c1 (beta1)."""
    grid: Grid
    trap: Trap = field(default_factory=Trap)
    Omega: float = 0.0
    gamma: float = 0.0
    c0: float = 0.0
    c1: float = 0.0

    def __post_init__(self):
        self.V = self.trap.values(self.grid)

    # ------------------------------------------------------------------ spectral pieces
    def spec(self, Phi):
        return fftn(Phi, self.grid.stack_axes)

    def ispec(self, Phat):
        return ifftn(Phat, self.grid.stack_axes)

    def derivs(self, Phi):
        """Spectral first derivatives d/dx_i and the Laplacian of every component.

        d/dx_i -> multiply coefficients by i v_i; Laplacian -> by -|v|^2
        (Section 3.2, symbols of Delta; first derivatives give L0, L1, Lz)."""
        Ph = self.spec(Phi)
        g = self.grid
        grads = [self.ispec(1j * g.K[i] * Ph) for i in range(g.d)]
        lap = self.ispec(-g.K2 * Ph)
        return grads, lap

    # ------------------------------------------------------------------ operators
    def Lz(self, Phi, grads=None):
        """Lz phi = -i (x d_y phi - y d_x phi) (Section 1, after Eq. GPE3)."""
        if grads is None:
            grads, _ = self.derivs(Phi)
        x, y = self.grid.X[0], self.grid.X[1]
        return -1j * (x * grads[1] - y * grads[0])

    def L0(self, phi, grads):
        """L0 = i d_x + d_y (Section 1); R-SOC3D."""
        return 1j * grads[0] + grads[1]

    def L1(self, phi, grads):
        """L1 = i d_x - d_y (Section 1); R-SOC3D."""
        return 1j * grads[0] - grads[1]

    def S_apply(self, Phi, grads=None):
        """S Phi with S = [[0, L0, 0], [L1, 0, L0], [0, L1, 0]] (Section 1)."""
        if grads is None:
            grads, _ = self.derivs(Phi)
        g = [[gr[c] for gr in grads] for c in range(3)]  # per component list of derivatives
        out = np.empty_like(Phi)
        out[0] = self.L0(Phi[1], g[1])
        out[1] = self.L1(Phi[0], g[0]) + self.L0(Phi[2], g[2])
        out[2] = self.L1(Phi[1], g[1])
        return out

    def H_lin(self, Phi, grads=None, lap=None):
        """Linear part -1/2 Laplacian + V - Omega Lz - gamma S applied to Phi."""
        if grads is None or lap is None:
            grads, lap = self.derivs(Phi)
        return (-0.5 * lap + self.V[None] * Phi - self.Omega * self.Lz(Phi, grads)
                - self.gamma * self.S_apply(Phi, grads))

    # ------------------------------------------------------------------ densities
    @staticmethod
    def densities(Phi):
        """rho_l = |phi_l|^2 and rho = sum (Section 1)."""
        rl = np.abs(Phi) ** 2
        return rl, rl.sum(axis=0)

    @staticmethod
    def spin_vector(Phi):
        """(F_x, F_y, F_z), explicit formulas of Section 1 (real fields)."""
        p1, p0, pm = Phi[0], Phi[1], Phi[2]
        c1, c0, cm = np.conj(p1), np.conj(p0), np.conj(pm)
        Fx = (c1 * p0 + c0 * (p1 + pm) + cm * p0) / SQ2
        Fy = 1j * (-c1 * p0 + c0 * (p1 - pm) + cm * p0) / SQ2
        Fz = np.abs(p1) ** 2 - np.abs(pm) ** 2
        return np.real(Fx), np.real(Fy), np.real(Fz)

    @staticmethod
    def Ff_apply(F, P):
        """(F . f) P with the 3x3 matrix of Section 1, F_pm = F_x +- i F_y."""
        Fx, Fy, Fz = F
        Fp = Fx + 1j * Fy
        Fm = Fx - 1j * Fy
        out = np.empty_like(P)
        out[0] = Fz * P[0] + Fm / SQ2 * P[1]
        out[1] = Fp / SQ2 * P[0] + Fm / SQ2 * P[2]
        out[2] = Fp / SQ2 * P[1] - Fz * P[2]
        return out

    # ------------------------------------------------------------------ H_l(Phi)
    def H(self, Phi, grads=None, lap=None):
        """H_l(Phi), l = 1, 0, -1, component form of Eqs. eigen1-eigen3.

        H0 phi = -1/2 Laplacian phi + V phi + c0 rho phi - Omega Lz phi."""
        if grads is None or lap is None:
            grads, lap = self.derivs(Phi)
        rl, rho = self.densities(Phi)
        p1, p0, pm = Phi[0], Phi[1], Phi[2]
        lz = self.Lz(Phi, grads)
        H0 = -0.5 * lap + (self.V + self.c0 * rho)[None] * Phi - self.Omega * lz
        g = [[gr[c] for gr in grads] for c in range(3)]
        c1, gam = self.c1, self.gamma
        out = np.empty_like(Phi)
        out[0] = (H0[0] + c1 * (rl[1] + rl[0] - rl[2]) * p1 + c1 * np.conj(pm) * p0 * p0
                  - gam * self.L0(p0, g[1]))
        out[1] = (H0[1] + c1 * (rl[0] + rl[2]) * p0 + 2.0 * c1 * pm * np.conj(p0) * p1
                  - gam * (self.L0(pm, g[2]) + self.L1(p1, g[0])))
        out[2] = (H0[2] + c1 * (rl[1] + rl[2] - rl[0]) * pm + c1 * p0 * p0 * np.conj(p1)
                  - gam * self.L1(p0, g[1]))
        return out

    def H_frozen(self, Phi, P):
        """R-FROZEN: [H_lin + c0 rho(Phi) + c1 F(Phi).f] P, the operator of Eq. an."""
        _, rho = self.densities(Phi)
        F = self.spin_vector(Phi)
        return self.H_lin(P) + self.c0 * rho[None] * P + self.c1 * self.Ff_apply(F, P)

    # ------------------------------------------------------------------ functionals
    def inner(self, v, u) -> complex:
        """<v, u> = integral sum_l v_l conj(u_l) (Section 2.2, after Eq. phase-factor)."""
        return complex(np.sum(v * np.conj(u))) * self.grid.dV

    def mass(self, Phi) -> float:
        """N(Phi) = integral sum_l |phi_l|^2 (Eq. mass)."""
        return self.grid.integrate(np.abs(Phi) ** 2)

    def masses(self, Phi):
        return [self.grid.integrate(np.abs(Phi[c]) ** 2) for c in range(3)]

    def energy_parts(self, Phi):
        """Pieces of Eq. energy: kinetic, potential, rotation, interaction (c0, c1), SOC."""
        grads, lap = self.derivs(Phi)
        g = self.grid
        kin = 0.5 * sum(g.integrate(np.abs(gr) ** 2) for gr in grads)
        pot = g.integrate(self.V[None] * np.abs(Phi) ** 2)
        rot = -self.Omega * g.integrate(np.conj(Phi) * self.Lz(Phi, grads))
        _, rho = self.densities(Phi)
        F = self.spin_vector(Phi)
        e_c0 = g.integrate(0.5 * self.c0 * rho * rho)
        e_c1 = g.integrate(0.5 * self.c1 * (F[0] ** 2 + F[1] ** 2 + F[2] ** 2))
        soc = -self.gamma * g.integrate(np.conj(Phi) * self.S_apply(Phi, grads))
        return dict(kin=kin, pot=pot, rot=rot, c0=e_c0, c1=e_c1, soc=soc,
                    spin=e_c0 + e_c1)

    def energy(self, Phi) -> float:
        """E(Phi) of Eq. energy, with the kinetic term written as
        integral conj(phi)(-1/2 Laplacian phi) on the grid."""
        grads, lap = self.derivs(Phi)
        g = self.grid
        _, rho = self.densities(Phi)
        F = self.spin_vector(Phi)
        lin = (-0.5 * lap + self.V[None] * Phi - self.Omega * self.Lz(Phi, grads))
        dens = np.sum(np.conj(Phi) * lin, axis=0)
        dens = dens + 0.5 * self.c0 * rho * rho + 0.5 * self.c1 * (F[0] ** 2 + F[1] ** 2 + F[2] ** 2)
        dens = dens - self.gamma * np.sum(np.conj(Phi) * self.S_apply(Phi, grads), axis=0)
        return g.integrate(dens)

    def energy_E2(self, Phi) -> float:
        """Interaction energy in the explicit form E2 of Section 2.1 (no F)."""
        p1, p0, pm = Phi[0], Phi[1], Phi[2]
        _, rho = self.densities(Phi)
        t1 = np.real((np.conj(p1) + np.conj(pm)) * p0) ** 2
        t2 = np.imag(p0 * (np.conj(pm) - np.conj(p1))) ** 2
        t3 = (np.abs(p1) ** 2 - np.abs(pm) ** 2) ** 2
        return self.grid.integrate(0.5 * self.c0 * rho * rho + 0.5 * self.c1 * (2 * t1 + 2 * t2 + t3))

    def mu(self, Phi, HPhi=None) -> float:
        """mu(Phi) = integral sum_l H_l(Phi) conj(phi_l) (Eq. muphi), real part."""
        if HPhi is None:
            HPhi = self.H(Phi)
        return self.inner(HPhi, Phi).real

    # ------------------------------------------------------------------ step model (Section 3.1)
    @staticmethod
    def Ftilde(v, u):
        """Conjugate bilinear forms F~_x, F~_y, F~_z(v, u) of Section 3.1."""
        u1, u0, um = np.conj(u[0]), np.conj(u[1]), np.conj(u[2])
        v1, v0, vm = v[0], v[1], v[2]
        fx = (u1 * v0 + u0 * (v1 + vm) + um * v0) / SQ2
        fy = 1j * (-u1 * v0 + u0 * (v1 - vm) + um * v0) / SQ2
        fz = u1 * v1 - um * vm
        return fx, fy, fz

    def step_coefficients(self, Phi, P, HPhi, mu):
        """a_n, b_n of Eqs. an, bn (R-FROZEN for H_l(P^n))."""
        nP2 = self.mass(P)
        nP = math.sqrt(nP2)
        HP = self.H_frozen(Phi, P)
        quad = self.inner(HP, P).real / nP2
        re_phiP = np.real(np.sum(np.conj(Phi) * P, axis=0))
        Ft = self.Ftilde(Phi, P)
        quart = self.grid.integrate(self.c0 * re_phiP ** 2
                                    + self.c1 * sum(np.real(f) ** 2 for f in Ft))
        a = -mu + quad + 2.0 * quart / nP2
        b = 2.0 / nP * self.inner(HPhi, P).real
        return a, b

    def energy_change(self, Phi, Phat, theta) -> float:
        """E(cos(theta) Phi + sin(theta) Phat) - E(Phi), written out in sin/cos
        (Section 3.1, the explicit trigonometric form of E(theta) after Eq. theta).

        With c = cos(theta), s = sin(theta) and c^2 - 1 = -s^2:
          quadratic part: -s^2 <H_lin Phi, Phi> + 2 c s Re<H_lin Phi, Phat> + s^2 <H_lin Phat, Phat>
          rho_t - rho = -s^2 rho_Phi + 2 c s Re(Phi^dag Phat) + s^2 rho_Phat
          F_t - F     = -s^2 F(Phi) + 2 c s Re F~(Phi, Phat) + s^2 F(Phat)
          interaction: c0/2 (rho_t - rho)(rho_t + rho) + c1/2 sum_alpha (F_t - F)(F_t + F).
        R-DE: the step-acceptance test and the stop3 difference use this form
        (no cancellation between two O(1) energies)."""
        c, s = math.cos(theta), math.sin(theta)
        HP = self.H_lin(Phat)
        HF = self.H_lin(Phi)
        quad = (-s * s * self.inner(HF, Phi).real + 2 * c * s * self.inner(HF, Phat).real
                + s * s * self.inner(HP, Phat).real)
        _, rf = self.densities(Phi)
        _, rp = self.densities(Phat)
        R = np.real(np.sum(np.conj(Phi) * Phat, axis=0))
        drho = -s * s * rf + 2 * c * s * R + s * s * rp
        Ff = self.spin_vector(Phi)
        Fp = self.spin_vector(Phat)
        Ft = self.Ftilde(Phi, Phat)
        inter = 0.5 * self.c0 * drho * (2 * rf + drho)
        for a in range(3):
            dF = -s * s * Ff[a] + 2 * c * s * np.real(Ft[a]) + s * s * Fp[a]
            inter = inter + 0.5 * self.c1 * dF * (2 * Ff[a] + dF)
        return quad + self.grid.integrate(inter)

    def trig_form(self, Phi, Phat):
        """E(cos(t) Phi + sin(t) Phat) - E(Phi) and its t-derivative as explicit functions of t
        (Section 3.1, the rewrite of E(theta) in sin and cos whose coefficients are integrals).

        With c = cos t, s = sin t the combination's coefficients are u = c^2 - 1 = -s^2 on the
        Phi-Phi terms, v = 2cs on the Phi-Phat cross terms and w = s^2 on the Phat-Phat terms:
          quadratic part  u <H_lin Phi, Phi> + v Re<H_lin Phi, Phat> + w <H_lin Phat, Phat>
          rho_t - rho     = u rho_Phi + v R + w rho_Phat,   R = Re sum_l conj(phi_l) phat_l
          F_t - F         = u F(Phi) + v Re F~(Phi, Phat) + w F(Phat)
          interaction     c0/2 int (rho_t - rho)(rho_t + rho) + c1/2 int (F_t - F).(F_t + F)
        so Delta E is a quadratic polynomial in (u, v, w) whose coefficients are integrals of
        Phi and Phat computed here once; du/dt = -sin 2t, dv/dt = 2 cos 2t, dw/dt = sin 2t.
        Returns (dE(t), dE'(t)) as functions of t."""
        g = self.grid
        HF, HP = self.H_lin(Phi), self.H_lin(Phat)
        l1 = {"u": self.inner(HF, Phi).real, "v": self.inner(HF, Phat).real, "w": self.inner(HP, Phat).real}
        _, rf = self.densities(Phi)
        _, rp = self.densities(Phat)
        R = np.real(np.sum(np.conj(Phi) * Phat, axis=0))
        dens = {"u": rf, "v": R, "w": rp}
        Ff, Fp, Fx = self.spin_vector(Phi), self.spin_vector(Phat), self.Ftilde(Phi, Phat)
        spin = {"u": Ff, "v": tuple(np.real(f) for f in Fx), "w": Fp}
        keys = ("u", "v", "w")
        # linear coefficient of each variable and the symmetric quadratic coefficients
        lin = {k: l1[k] + self.c0 * g.integrate(rf * dens[k])
               + self.c1 * g.integrate(sum(Ff[a] * spin[k][a] for a in range(3))) for k in keys}
        quad = {(i, j): 0.5 * self.c0 * g.integrate(dens[i] * dens[j])
                + 0.5 * self.c1 * g.integrate(sum(spin[i][a] * spin[j][a] for a in range(3)))
                for i in keys for j in keys}

        def parts(t):
            c, s = math.cos(t), math.sin(t)
            x = {"u": -s * s, "v": 2 * c * s, "w": s * s}
            dx = {"u": -math.sin(2 * t), "v": 2 * math.cos(2 * t), "w": math.sin(2 * t)}
            return x, dx

        def dE(t):
            x, _ = parts(t)
            return (sum(lin[k] * x[k] for k in keys)
                    + sum(quad[(i, j)] * x[i] * x[j] for i in keys for j in keys))

        def dE1(t):
            x, dx = parts(t)
            return (sum(lin[k] * dx[k] for k in keys)
                    + sum(quad[(i, j)] * (dx[i] * x[j] + x[i] * dx[j]) for i in keys for j in keys))
        return dE, dE1

    # ------------------------------------------------------------------ preconditioners (Section 3.4)
    def alpha(self, Phi):
        """alpha_l = integral 1/2|grad phi_l|^2 + V|phi_l|^2 + c0 rho |phi_l|^2 (Eq. PreCnstAlpha), R-ALPHA."""
        grads, _ = self.derivs(Phi)
        _, rho = self.densities(Phi)
        g = self.grid
        al = []
        for c in range(3):
            kin = 0.5 * sum(g.integrate(np.abs(gr[c]) ** 2) for gr in grads)
            al.append(kin + g.integrate((self.V + self.c0 * rho) * np.abs(Phi[c]) ** 2))
        floor = 1e-12 * max(abs(a) for a in al) + 1e-300
        return [max(a, floor) for a in al]

    def precond_V_sqrt(self, Phi, alpha):
        """Diagonal of P_V^{1/2}: 1/sqrt(alpha_l + V + c0 rho) (Eq. PreCondPot), R-ALPHA."""
        _, rho = self.densities(Phi)
        out = []
        for c in range(3):
            den = alpha[c] + self.V + self.c0 * rho
            den = np.maximum(den, 1e-12 * alpha[c])
            out.append(1.0 / np.sqrt(den))
        return np.stack(out)

    def precond_Delta(self, W, alpha):
        """P_Delta W: divide coefficient k of component l by alpha_l + |v|^2/2 (Eq. PreCondKin)."""
        Wh = self.spec(W)
        den = np.stack([alpha[c] + 0.5 * self.grid.K2 for c in range(3)])
        return self.ispec(Wh / den)

    def precond_C(self, r, Phi, alpha):
        """P_C = P_V^{1/2} P_Delta P_V^{1/2} (Eq. PreCondMix)."""
        s = self.precond_V_sqrt(Phi, alpha)
        return s * self.precond_Delta(s * r, alpha)

    def precond_kin(self, r, Phi, alpha):
        """P_Delta alone (Eq. PreCondKin)."""
        return self.precond_Delta(r, alpha)

    def precond_pot(self, r, Phi, alpha):
        """P_V alone (Eq. PreCondPot)."""
        s = self.precond_V_sqrt(Phi, alpha)
        return s * s * r

    # ------------------------------------------------------------------ diagnostics
    def virial(self, Phi) -> float:
        """I = 2 E_kin - 2 E_pot + d E_spin + E_soc (Eq. virial; harmonic V)."""
        e = self.energy_parts(Phi)
        return 2 * e["kin"] - 2 * e["pot"] + self.grid.d * e["spin"] + e["soc"]


def phase_align(Phi1, Phi2, model: Model):
    """kappa = <Phi1, Phi2>/<Phi2, Phi2> (Eq. phase-factor); returns conj(kappa) Phi1
    normalised to unit modulus phase, for gauge-invariant comparison with Phi2."""
    kappa = model.inner(Phi1, Phi2) / model.inner(Phi2, Phi2)
    ph = kappa / abs(kappa) if abs(kappa) > 0 else 1.0
    return np.conj(ph) * Phi1, kappa
