"""Pins of the oracle's discrete model against closed forms, definitions typed
independently from the paper's other formulas, and calculus identities."""
import math

import numpy as np
import pytest

import seeded_inputs as si
from oracle.model import Grid, Model, Trap

SQ2 = math.sqrt(2.0)


def _model(n=(32, 32), L=(6.0, 6.0), **kw):
    g = Grid(n, L)
    return Model(g, kw.pop("trap", Trap()), **kw)


def _smooth(m, seed, width=1.2):
    return si.smooth_random_state(m.grid.n, m.grid.L, seed, width)


def test_grid_coordinates_and_wavenumbers():
    g = Grid((8, 4), (2.0, 3.0))
    np.testing.assert_allclose(g.X[0].ravel(), -2.0 + 0.5 * np.arange(8))
    np.testing.assert_allclose(g.X[1].ravel(), -3.0 + 1.5 * np.arange(4))
    # v_p = pi p / L with p = 0..N/2-1, -N/2..-1 in index order (Section 3.2)
    np.testing.assert_allclose(g.K[0].ravel(), math.pi / 2.0 * np.array([0, 1, 2, 3, -4, -3, -2, -1]))
    assert g.dV == 0.5 * 1.5


def test_plane_wave_derivatives_and_soc_operators():
    # phi = exp(i(a x + b y)) with a, b on the grid's wavenumber lattice:
    # d_x phi = i a phi; L0 = i d_x + d_y -> (-a + i b); L1 = i d_x - d_y -> (-a - i b)
    m = _model((16, 16), (4.0, 4.0))
    a, b = math.pi * 3 / 4.0, -math.pi * 2 / 4.0
    X, Y = m.grid.X
    phi = np.exp(1j * (a * X + b * Y)) * np.ones(m.grid.shape)
    Phi = np.stack([phi, 2 * phi, -phi])
    grads, lap = m.derivs(Phi)
    np.testing.assert_allclose(grads[0], 1j * a * Phi, atol=1e-12)
    np.testing.assert_allclose(grads[1], 1j * b * Phi, atol=1e-12)
    np.testing.assert_allclose(lap, -(a * a + b * b) * Phi, atol=1e-11)
    g0 = [gr[1] for gr in grads]
    np.testing.assert_allclose(m.L0(Phi[1], g0), (-a + 1j * b) * Phi[1], atol=1e-12)
    np.testing.assert_allclose(m.L1(Phi[1], g0), (-a - 1j * b) * Phi[1], atol=1e-12)


def test_lz_eigenfunctions():
    # Lz = -i(x d_y - y d_x): (x + i y) e^{-r^2/2} has eigenvalue +1, (x - i y) e^{-r^2/2} has -1,
    # a radial function has 0.
    m = _model((64, 64), (8.0, 8.0))
    X, Y = m.grid.X
    g = np.exp(-(X * X + Y * Y) / 2)
    Phi = np.stack([(X + 1j * Y) * g, (X - 1j * Y) * g, g + 0j])
    lz = m.Lz(Phi)
    np.testing.assert_allclose(lz[0], Phi[0], atol=1e-12)
    np.testing.assert_allclose(lz[1], -Phi[1], atol=1e-12)
    np.testing.assert_allclose(lz[2], 0 * Phi[2], atol=1e-12)


def test_gaussian_laplacian_closed_form():
    m = _model((64, 64), (8.0, 8.0))
    X, Y = m.grid.X
    r2 = X * X + Y * Y
    g = np.exp(-r2 / 2)
    _, lap = m.derivs(np.stack([g + 0j] * 3))
    np.testing.assert_allclose(lap[0], (r2 - 2) * g, atol=1e-11)


def test_spin_vector_matches_matrix_definition():
    # F_alpha = Psi^dagger f_alpha Psi with the spin-1 matrices of Section 1
    fx = np.array([[0, 1, 0], [1, 0, 1], [0, 1, 0]]) / SQ2
    fy = 1j * np.array([[0, -1, 0], [1, 0, -1], [0, 1, 0]]) / SQ2
    fz = np.diag([1.0, 0.0, -1.0])
    m = _model((8, 8), (3.0, 3.0))
    Phi = si.random_state(m.grid.n, 11)
    F = m.spin_vector(Phi)
    for f, Fa in zip((fx, fy, fz), F):
        ref = np.einsum("i...,ij,j...->...", np.conj(Phi), f, Phi)
        assert np.max(np.abs(ref.imag)) < 1e-13  # Hermitian matrices give real F
        np.testing.assert_allclose(Fa, ref.real, atol=1e-13)
    # F.f matrix of Section 1 equals sum_alpha F_alpha f_alpha
    Ff = m.Ff_apply(F, Phi)
    ref = sum(Fa[None] * np.einsum("ij,j...->i...", f, Phi) for f, Fa in zip((fx, fy, fz), F))
    np.testing.assert_allclose(Ff, ref, atol=1e-13)


def test_interaction_energy_E2_form():
    # E2 of Section 2.1 (no F) equals integral c0/2 rho^2 + c1/2 |F|^2
    m = _model((16, 16), (4.0, 4.0), c0=3.0, c1=-1.7)
    Phi = si.random_state(m.grid.n, 5)
    parts = m.energy_parts(Phi)
    assert m.energy_E2(Phi) == pytest.approx(parts["c0"] + parts["c1"], rel=1e-13)


def test_energy_is_sum_of_parts_and_phase_invariant():
    m = _model((32, 32), (6.0, 6.0), Omega=0.4, gamma=0.7, c0=20.0, c1=-2.0)
    Phi = _smooth(m, 1)
    e = m.energy_parts(Phi)
    total = e["kin"] + e["pot"] + e["rot"] + e["c0"] + e["c1"] + e["soc"]
    assert m.energy(Phi) == pytest.approx(total, rel=1e-12)
    kappa = np.exp(0.73j)
    assert m.energy(kappa * Phi) == pytest.approx(m.energy(Phi), rel=1e-13)


def _dense(op, shape):
    n = int(np.prod(shape))
    A = np.empty((n, n), dtype=np.complex128)
    for j in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[j] = 1.0
        A[:, j] = op(e.reshape(shape)).ravel()
    return A


def test_linear_operator_hermitian_and_soc_symbol():
    m = _model((8, 8), (3.0, 3.0), Omega=0.7, gamma=0.9)
    shape = (3,) + m.grid.shape
    A = _dense(m.H_lin, shape)
    assert np.max(np.abs(A - A.conj().T)) < 1e-12 * np.max(np.abs(A))
    # S on plane waves: the 3x3 symbol has eigenvalues {0, +-sqrt(2)|k_perp|}
    X, Y = m.grid.X
    kx, ky = math.pi * 2 / 3.0, math.pi * -1 / 3.0
    pw = np.exp(1j * (kx * X + ky * Y)) * np.ones(m.grid.shape)
    sym = np.zeros((3, 3), complex)
    for j in range(3):
        Phi = np.zeros(shape, complex)
        Phi[j] = pw
        out = m.S_apply(Phi)
        sym[:, j] = (out[:, 0, 0] / pw[0, 0])
    ev = np.sort(np.linalg.eigvals(sym).real)
    k = math.hypot(kx, ky)
    np.testing.assert_allclose(ev, [-SQ2 * k, 0.0, SQ2 * k], atol=1e-12)


def test_energy_gradient_is_H():
    # d/de E(Phi + e W) at e=0 equals 2 Re <H(Phi), W> (Euler-Lagrange, Eqs. eigen1-3).
    # E(Phi + eW) is a quartic in e: Richardson on central differences is exact up to rounding.
    m = _model((32, 32), (6.0, 6.0), Omega=0.45, gamma=0.8, c0=15.0, c1=-3.0)
    Phi = _smooth(m, 2)
    W = _smooth(m, 3)
    E = lambda e: m.energy(Phi + e * W)
    eps = 1e-3
    D1 = (E(eps) - E(-eps)) / (2 * eps)
    D2 = (E(2 * eps) - E(-2 * eps)) / (4 * eps)
    deriv = (4 * D1 - D2) / 3
    grad = 2 * m.inner(m.H(Phi), W).real
    assert deriv == pytest.approx(grad, rel=2e-8)
    # the same for each parameter switched on alone (catches a term typed into only one side)
    for kw in (dict(Omega=0.6), dict(gamma=1.1), dict(c0=30.0), dict(c1=7.0)):
        mm = _model((32, 32), (6.0, 6.0), **kw)
        Em = lambda e: mm.energy(Phi + e * W)
        D1 = (Em(eps) - Em(-eps)) / (2 * eps)
        D2 = (Em(2 * eps) - Em(-2 * eps)) / (4 * eps)
        assert (4 * D1 - D2) / 3 == pytest.approx(2 * mm.inner(mm.H(Phi), W).real, rel=2e-8), kw


def test_frozen_operator_on_phi_is_H():
    # [H_lin + c0 rho + c1 F.f] Phi equals the component form H(Phi) (Section 1 compact form)
    m = _model((16, 16), (4.0, 4.0), Omega=0.3, gamma=0.6, c0=9.0, c1=-2.5)
    Phi = _smooth(m, 4)
    np.testing.assert_allclose(m.H_frozen(Phi, Phi), m.H(Phi), atol=1e-12)


def test_mu_energy_identity_and_orthogonality():
    # mu = E + integral c0/2 rho^2 + c1/2 |F|^2 ; Re <Phi, r> = 0 for ||Phi|| = 1
    m = _model((32, 32), (6.0, 6.0), Omega=0.5, gamma=0.4, c0=40.0, c1=1.5)
    Phi = _smooth(m, 6)
    Phi = Phi / math.sqrt(m.mass(Phi))
    e = m.energy_parts(Phi)
    H = m.H(Phi)
    mu = m.mu(Phi, H)
    assert mu == pytest.approx(m.energy(Phi) + e["c0"] + e["c1"], rel=1e-12)
    r = H - mu * Phi
    assert abs(m.inner(Phi, r).real) < 1e-12 * abs(mu)


def test_step_coefficients_are_derivatives_of_energy_along_the_sphere():
    # b_n = E'(0), 2 a_n = E''(0) for E(theta) = E(cos(theta) Phi + sin(theta) P/||P||) (Eqs. approeng-bn)
    m = _model((32, 32), (6.0, 6.0), Omega=0.55, gamma=0.9, c0=25.0, c1=-4.0)
    Phi = _smooth(m, 8)
    Phi = Phi / math.sqrt(m.mass(Phi))
    D = _smooth(m, 9)
    P = D - m.inner(D, Phi).real * Phi
    assert abs(m.inner(P, Phi).real) < 1e-13
    H = m.H(Phi)
    mu = m.mu(Phi, H)
    a, b = m.step_coefficients(Phi, P, H, mu)
    Ph = P / math.sqrt(m.mass(P))
    E = lambda t: m.energy(math.cos(t) * Phi + math.sin(t) * Ph)
    h = 1e-3
    d1 = [(E(s * h) - E(-s * h)) / (2 * s * h) for s in (1, 2)]
    d2 = [(E(s * h) - 2 * E(0) + E(-s * h)) / (s * h) ** 2 for s in (1, 2)]
    E1 = (4 * d1[0] - d1[1]) / 3
    E2 = (4 * d2[0] - d2[1]) / 3
    assert b == pytest.approx(E1, rel=1e-7)
    assert 2 * a == pytest.approx(E2, rel=1e-5)


def test_psd_direction_has_negative_slope():
    # With beta = 0, D = -P r and b_n = -2 Re<P r, r>/||P|| < 0 (Section 3.1, after Eq. bn)
    m = _model((32, 32), (6.0, 6.0), Omega=0.5, gamma=0.5, c0=30.0, c1=-1.0)
    Phi = _smooth(m, 10)
    Phi = Phi / math.sqrt(m.mass(Phi))
    H = m.H(Phi)
    mu = m.mu(Phi, H)
    r = H - mu * Phi
    al = m.alpha(Phi)
    Pr = m.precond_C(r, Phi, al)
    D = -Pr
    P = D - m.inner(D, Phi).real * Phi
    a, b = m.step_coefficients(Phi, P, H, mu)
    assert b < 0
    assert b == pytest.approx(-2 * m.inner(Pr, r).real / math.sqrt(m.mass(P)), rel=1e-10)


def test_preconditioners_symmetric_positive_definite():
    m = _model((16, 16), (4.0, 4.0), Omega=0.3, gamma=0.3, c0=50.0, c1=1.0)
    Phi = _smooth(m, 12)
    Phi = Phi / math.sqrt(m.mass(Phi))
    al = m.alpha(Phi)
    assert min(al) > 0
    x = si.random_state(m.grid.n, 13)
    y = si.random_state(m.grid.n, 14)
    for op in (m.precond_C, m.precond_kin, m.precond_pot):
        px, py = op(x, Phi, al), op(y, Phi, al)
        assert m.inner(x, py) == pytest.approx(np.conj(m.inner(y, px)), rel=1e-12)
        assert m.inner(px, x).real > 0


def test_alpha_matches_definition_pieces():
    # alpha_l = kinetic_l + potential_l + c0 integral rho |phi_l|^2 (Eq. PreCnstAlpha); kinetic via
    # -1/2 integral conj(phi) Laplacian phi (summation by parts on the periodic grid)
    m = _model((32, 32), (6.0, 6.0), c0=12.0)
    Phi = _smooth(m, 15)
    _, lap = m.derivs(Phi)
    _, rho = m.densities(Phi)
    al = m.alpha(Phi)
    for c in range(3):
        kin = m.grid.integrate(-0.5 * np.conj(Phi[c]) * lap[c])
        ref = kin + m.grid.integrate((m.V + 12.0 * rho) * np.abs(Phi[c]) ** 2)
        assert al[c] == pytest.approx(ref, rel=1e-12)


def test_energy_change_expansion_matches_direct_difference():
    # explicit sin/cos form of E(theta) - E(0) (Section 3.1) vs two direct energy evaluations
    m = _model((32, 32), (6.0, 6.0), Omega=0.55, gamma=0.9, c0=25.0, c1=-4.0)
    Phi = _smooth(m, 16)
    Phi = Phi / math.sqrt(m.mass(Phi))
    D = _smooth(m, 17)
    P = D - m.inner(D, Phi).real * Phi
    Ph = P / math.sqrt(m.mass(P))
    E0 = m.energy(Phi)
    for t in (1.3, 0.4, 0.05, 1e-3):
        direct = m.energy(math.cos(t) * Phi + math.sin(t) * Ph) - E0
        assert m.energy_change(Phi, Ph, t) == pytest.approx(direct, rel=1e-9, abs=1e-12)


# ---------------------------------------------------------------- preconditioners pinned in closed form
def _plane_waves(m, waves, amps=(1.0, 1.0, 1.0)):
    """Component l = amps[l] exp(i k_l . x) with k_l on the grid's wavenumber lattice
    (waves[l] = integer multiples of pi/L_i per axis)."""
    g = m.grid
    out = []
    for c in range(3):
        ph = sum(math.pi * waves[c][i] / g.L[i] * g.X[i] for i in range(g.d))
        out.append(amps[c] * np.exp(1j * ph) * np.ones(g.shape))
    return np.stack(out)


@pytest.mark.parametrize("n,L", [((16, 16), (4.0, 4.0)), ((8, 16, 8), (3.0, 4.0, 2.5))])
def test_kinetic_preconditioner_divides_plane_waves_by_alpha_plus_half_k2(n, L):
    # P_Delta (Eq. PreCondKin) is the Fourier multiplier 1/(alpha_l + |k|^2/2): a plane wave
    # exp(i k.x) in component l comes back scaled by exactly that factor
    m = _model(n, L)
    d = len(n)
    waves = [(3, -2, 1)[:d], (0, 5, -3)[:d], (-4, 1, 2)[:d]]
    W = _plane_waves(m, waves, (1.0, 0.5 - 0.3j, 2.0))
    alpha = [0.7, 1.3, 2.1]
    out = m.precond_Delta(W, alpha)
    for c in range(3):
        k2 = sum((math.pi * waves[c][i] / L[i]) ** 2 for i in range(d))
        np.testing.assert_allclose(out[c], W[c] / (alpha[c] + 0.5 * k2), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(m.precond_kin(W, W, alpha), out, rtol=1e-14, atol=1e-16)


def test_potential_preconditioner_is_pointwise_inverse_of_alpha_plus_V_plus_c0_rho():
    # P_V (Eq. PreCondPot) multiplies component l by 1/(alpha_l + V + c0 rho); the square-root
    # factor of P_C by 1/sqrt(alpha_l + V + c0 rho); V = (gx^2 x^2 + gy^2 y^2)/2 typed here
    c0 = 7.5
    m = _model((16, 16), (4.0, 4.0), trap=Trap(g=(1.0, 1.7)), c0=c0)
    X, Y = m.grid.X
    V = 0.5 * (X * X + (1.7 * Y) ** 2)
    Phi = _smooth(m, 31)
    rho = sum(np.abs(Phi[c]) ** 2 for c in range(3))
    r = si.random_state(m.grid.n, 32)
    alpha = [0.4, 0.9, 3.2]
    s = m.precond_V_sqrt(Phi, alpha)
    pot = m.precond_pot(r, Phi, alpha)
    for c in range(3):
        den = alpha[c] + V + c0 * rho
        np.testing.assert_allclose(s[c], 1.0 / np.sqrt(den), rtol=1e-14)
        np.testing.assert_allclose(pot[c], r[c] / den, rtol=1e-13)


@pytest.mark.parametrize("n,L", [((16, 16), (4.0, 4.0)), ((8, 8, 16), (3.0, 3.0, 4.0))])
def test_combined_preconditioner_and_alpha_closed_form_on_uniform_density(n, L):
    # V = 0 and plane-wave components a_l exp(i k_l.x): rho = sum |a_l|^2 is constant, so
    #   alpha_l = |a_l|^2 |D| (|k_l|^2/2 + c0 rho)       (Eq. PreCnstAlpha, |D| = prod 2 L_i)
    #   P_C exp(i q.x) e_l = exp(i q.x) e_l / ((alpha_l + c0 rho)(alpha_l + |q|^2/2))   (Eq. PreCondMix)
    # (each half of P_V^{1/2} contributes (alpha_l + c0 rho)^{-1/2}; P_Delta the kinetic factor)
    c0 = 3.0
    d = len(n)
    m = _model(n, L, trap=Trap(g=(0.0, 0.0, 0.0)), c0=c0, c1=-1.0, Omega=0.2, gamma=0.4)
    amps = (0.6, 0.3 + 0.2j, 0.25)
    kw = [(1, 2, 1)[:d], (-2, 0, 1)[:d], (0, -1, -2)[:d]]
    Phi = _plane_waves(m, kw, amps)
    rho = sum(abs(a) ** 2 for a in amps)
    vol = float(np.prod([2 * Li for Li in L]))
    alpha = m.alpha(Phi)
    for c in range(3):
        k2 = sum((math.pi * kw[c][i] / L[i]) ** 2 for i in range(d))
        assert alpha[c] == pytest.approx(abs(amps[c]) ** 2 * vol * (0.5 * k2 + c0 * rho), rel=1e-12)
    qw = [(3, -1, 2)[:d], (0, 4, -1)[:d], (-2, -3, 1)[:d]]
    r = _plane_waves(m, qw, (1.0, -0.7j, 0.4))
    z = m.precond_C(r, Phi, alpha)
    for c in range(3):
        q2 = sum((math.pi * qw[c][i] / L[i]) ** 2 for i in range(d))
        fac = 1.0 / ((alpha[c] + c0 * rho) * (alpha[c] + 0.5 * q2))
        np.testing.assert_allclose(z[c], fac * r[c], rtol=1e-12, atol=1e-15)


def test_trig_form_is_the_energy_change_and_its_derivative():
    # Section 3.1: E(cos t Phi + sin t Phat) - E(Phi) written out in sin/cos with precomputed
    # integrals equals the direct difference of two energies; its derivative equals the finite
    # difference of the direct form and, at t = 0, the slope 2 Re<H(Phi), Phat>
    m = _model((32, 32), (6.0, 6.0), Omega=0.55, gamma=0.9, c0=25.0, c1=-4.0)
    Phi = _smooth(m, 16)
    Phi = Phi / math.sqrt(m.mass(Phi))
    D = _smooth(m, 17)
    P = D - m.inner(D, Phi).real * Phi
    Ph = P / math.sqrt(m.mass(P))
    dE, dE1 = m.trig_form(Phi, Ph)
    E0 = m.energy(Phi)
    for t in (2.9, 1.3, 0.4, 0.05):
        direct = m.energy(math.cos(t) * Phi + math.sin(t) * Ph) - E0
        assert dE(t) == pytest.approx(direct, rel=1e-9, abs=1e-12)
        h = 1e-4
        fd = (m.energy_change(Phi, Ph, t + h) - m.energy_change(Phi, Ph, t - h)) / (2 * h)
        assert dE1(t) == pytest.approx(fd, rel=1e-6, abs=1e-9)
    assert dE1(0.0) == pytest.approx(2 * m.inner(m.H(Phi), Ph).real, rel=1e-12)
    assert dE(math.pi) == pytest.approx(0.0, abs=1e-12)            # period pi: E(-Phi) = E(Phi)


def test_exact_theta_minimises_the_energy_along_the_curve():
    # Eq. theta: the exact step is a stationary point with lower energy than the quadratic
    # model's step and than its neighbours
    from oracle.pcg import exact_theta
    m = _model((32, 32), (6.0, 6.0), Omega=0.5, gamma=0.5, c0=100.0, c1=-1.0)
    Phi = _smooth(m, 20)
    Phi = Phi / math.sqrt(m.mass(Phi))
    H = m.H(Phi)
    mu = m.mu(Phi, H)
    r = H - mu * Phi
    Pr = m.precond_C(r, Phi, m.alpha(Phi))
    P = -Pr - m.inner(-Pr, Phi).real * Phi
    a, b = m.step_coefficients(Phi, P, H, mu)
    Ph = P / math.sqrt(m.mass(P))
    assert b < 0
    tq = -b / (2 * a) if a > 0 else 0.1          # Algorithm 2's starting step
    t = exact_theta(m, Phi, Ph, tq)
    assert t > 0
    dE, dE1 = m.trig_form(Phi, Ph)
    assert abs(dE1(t)) < 1e-10 * abs(dE1(0.0))
    assert dE(t) <= dE(tq) + 1e-15
    for s in (0.9, 1.1):
        assert dE(t) < dE(s * t)
