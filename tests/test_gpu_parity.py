"""GPU parity: every step of the hot path through the C ABI against the FP64 oracle.

Tolerances (FP64 path): operator outputs within 1e-11 of the oracle's max
magnitude (FFT rounding grows like eps * log2(N) per transform, a few
transforms per operator); scalar reductions (E, mu, alpha, masses, a_n, b_n)
within 1e-12 relative; converged ground states: E and mu within 1e-10 relative,
densities and component masses within 1e-8 in max norm (BASELINE targets)."""
import math

import numpy as np
import pytest

import seeded_inputs as si
from oracle import guesses
from oracle.fft import fft_axis
from oracle.model import Grid, Model, Trap
from oracle.pcg import Options, cm_pcg, pcg, prolong
from tests.gpu_common import oracle_model, rel_max

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_17950_gb300 import build
    build.build()


from paper_2602_17950_gb300 import Problem  # noqa: E402

PAR = (0.45, 0.8, 30.0, -4.0)
GRIDS_2D = [((64, 64), (8.0, 8.0)), ((32, 64), (6.0, 9.0)), ((8, 16), (3.0, 4.0))]
GRIDS_3D = [((16, 16, 16), (5.0, 5.0, 5.0)), ((8, 16, 32), (4.0, 5.0, 6.0))]


@pytest.mark.parametrize("n,L", GRIDS_2D + GRIDS_3D)
def test_fft_axis_matches_oracle_fft(n, L):
    data = si.random_state(n, 3)[None].repeat(2, axis=0)  # two stacks of 3 components
    with Problem(n, L, [PAR, PAR]) as p:
        for axis in range(len(n)):
            for inverse in (False, True):
                t = torch.from_numpy(data.copy()).cuda()
                p.fft_axis(t.data_ptr(), 6, axis, inverse)
                got = t.cpu().numpy()
                ref = fft_axis(data, -1 - axis, inverse=inverse)
                assert rel_max(got, ref) < 1e-13 * math.log2(n[axis]) + 1e-15


@pytest.mark.parametrize("n,L", GRIDS_2D + GRIDS_3D)
def test_apply_h_matches_oracle(n, L):
    pars = [PAR, (0.0, 1.3, 0.0, 2.0), (0.9, 0.0, 200.0, 0.0)]
    psi = np.stack([si.smooth_random_state(n, L, 10 + k, width=min(L) / 3) for k in range(3)])
    trap = {"kind": 1, "g": (1.0, 1.3, 0.7), "quad": -0.2, "quart": 0.05}
    with Problem(n, L, pars, trap=trap) as p:
        p.set_initial(psi)
        hp, obs = p.apply_h()
        got_psi = p.psi()
    for k, par in enumerate(pars):
        m = oracle_model(n, L, par, trap)
        phi = got_psi[k]
        assert abs(m.mass(phi) - 1.0) < 1e-13
        H = m.H(phi)
        assert rel_max(hp[k], H) < 1e-11
        E, mu = m.energy(phi), m.mu(phi, H)
        al = m.alpha(phi)
        assert obs[k, 0] == pytest.approx(E, rel=1e-12)
        assert obs[k, 1] == pytest.approx(mu, rel=1e-12)
        np.testing.assert_allclose(obs[k, 2:5], al, rtol=1e-12)
        np.testing.assert_allclose(obs[k, 5:8], m.masses(phi), rtol=1e-12, atol=1e-15)
        assert obs[k, 8] == pytest.approx(m.inner(m.H_lin(phi), phi).real, rel=1e-12)


def test_user_potential_matches_oracle():
    n, L = (32, 32), (6.0, 6.0)
    X, Y = si.mesh(n, L)
    V = 0.3 * np.cos(X) * np.sin(0.5 * Y) + 0.1 * X
    trap = {"kind": 2, "g": (1.0, 1.0), "user_V": V}
    psi = si.smooth_random_state(n, L, 4)[None]
    with Problem(n, L, [PAR], trap=trap) as p:
        p.set_initial(psi)
        hp, obs = p.apply_h()
        phi = p.psi()[0]
    m = oracle_model(n, L, PAR, trap)
    assert rel_max(hp[0], m.H(phi)) < 1e-11
    assert obs[0, 0] == pytest.approx(m.energy(phi), rel=1e-12)


@pytest.mark.parametrize("n,L", [GRIDS_2D[0], GRIDS_2D[1], GRIDS_3D[1]])
def test_preconditioner_matches_oracle(n, L):
    psi = si.smooth_random_state(n, L, 21, width=min(L) / 3)[None]
    r = si.random_state(n, 22)[None]
    with Problem(n, L, [PAR]) as p:
        p.set_initial(psi)
        z = p.apply_precond(r)
        phi = p.psi()[0]
    m = oracle_model(n, L, PAR)
    al = m.alpha(phi)
    assert rel_max(z[0], m.precond_C(r[0], phi, al)) < 1e-11


@pytest.mark.parametrize("n,L", [GRIDS_2D[0], GRIDS_3D[0]])
def test_step_model_matches_oracle(n, L):
    psi = si.smooth_random_state(n, L, 31, width=min(L) / 3)[None]
    D = si.smooth_random_state(n, L, 32, width=min(L) / 3)
    thetas = np.array([1.2, 0.3, 1e-2, 1e-5])
    with Problem(n, L, [PAR]) as p:
        p.set_initial(psi)
        phi = p.psi()[0]
        m = oracle_model(n, L, PAR)
        P = D - m.inner(D, phi).real * phi
        out = p.step_model(P[None], thetas)
    H = m.H(phi)
    a, b = m.step_coefficients(phi, P, H, m.mu(phi, H))
    assert out[0, 0] == pytest.approx(a, rel=1e-11)
    assert out[0, 1] == pytest.approx(b, rel=1e-11)
    Ph = P / math.sqrt(m.mass(P))
    for k, t in enumerate(thetas):
        ref = m.energy_change(phi, Ph, t)
        assert out[0, 2 + k] == pytest.approx(ref, rel=1e-9, abs=1e-14 * abs(m.energy(phi)))


@pytest.mark.parametrize("n,L", [((32, 32), (6.0, 6.0)), ((16, 16, 32), (4.0, 4.0, 5.0))])
def test_prolongation_matches_oracle(n, L):
    coarse = tuple(k // 2 for k in n)
    psi = si.smooth_random_state(coarse, L, 41, width=min(L) / 3)[None]
    with Problem(n, L, [PAR]) as p:
        p.set_initial(psi, level=1)
        phic = p.psi()[0]
        p.prolong()
        fine = p.psi()[0]
    gc, gf = Grid(coarse, L), Grid(n, L)
    ref = prolong(phic, gc, gf)
    ref = ref / math.sqrt(Model(gf).mass(ref))
    assert rel_max(fine, ref) < 1e-12


def test_initial_guesses_match_oracle():
    n, L = (64, 64), (8.0, 8.0)
    par = (0.35, 0.5, 100.0, -1.0)
    m = oracle_model(n, L, par)
    for kinds in ([0, 1, 2], [3, 4, 5], [6, 7, 8], [9, 9, 0]):
        with Problem(n, L, [par]) as p:
            p.set_initial_kind(kinds)
            got = p.psi()[0]
        ref = guesses.spin1(m, kinds)
        ref = ref / math.sqrt(m.mass(ref))
        assert rel_max(got, ref) < 1e-12, kinds


def test_iterations_follow_oracle_step_by_step():
    # exactly 6 PCG iterations from the same seeded input: same trajectory
    n, L = (64, 64), (8.0, 8.0)
    par = (0.5, 0.5, 100.0, -1.0)
    psi0 = si.gaussian_guess(n, L, si.seed_for(1, 0))
    m = oracle_model(n, L, par)
    ref = pcg(m, psi0, Options(tol=1e-300, max_iter=6))
    assert ref.iters == 6
    with Problem(n, L, [par]) as p:
        p.set_initial(psi0[None])
        res = p.iterate(6)[0]
        got = p.psi()[0]
    assert res["iters"] == 6
    assert rel_max(got, ref.Phi) < 1e-9
    assert res["energy"] == pytest.approx(ref.energies[-2], rel=1e-12)  # E of the 6th iterate's start


def _solve_pair(n, L, par, psi0, tol=1e-12, res_tol=1e-9, trap=None):
    m = oracle_model(n, L, par, trap)
    ref = pcg(m, psi0, Options(tol=tol, res_tol=res_tol))
    with Problem(n, L, [par], trap=trap) as p:
        p.set_initial(psi0[None])
        res = p.solve(tol=tol, res_tol=res_tol)[0]
        got = p.psi()[0]
    return m, ref, res, got


def _assert_ground_state_parity(m, ref, res, got):
    assert ref.status == "converged" and res["status"] == "OK", res
    assert res["energy"] == pytest.approx(ref.energy, rel=1e-10)
    assert res["mu"] == pytest.approx(ref.mu, rel=1e-10)
    rho, rho_ref = np.abs(got) ** 2, np.abs(ref.Phi) ** 2
    assert np.max(np.abs(rho - rho_ref)) < 1e-8
    np.testing.assert_allclose(res["mass"], ref.masses, atol=1e-8)
    # the GPU's reported observables are those of its own final state
    assert res["energy"] == pytest.approx(m.energy(got), rel=1e-12)


def test_config1_ground_state_matches_oracle():
    # 64x64 on [-8,8]^2, Omega = 0.5, gamma = 0.5, beta0 = 100, beta1 = -1, seeded Gaussian
    n, L, par = (64, 64), (8.0, 8.0), (0.5, 0.5, 100.0, -1.0)
    psi0 = si.gaussian_guess(n, L, si.seed_for(1, 0))
    _assert_ground_state_parity(*_solve_pair(n, L, par, psi0))


def test_ragged_grid_ground_state_matches_oracle():
    n, L, par = (32, 64), (6.0, 10.0), (0.3, 0.9, 40.0, 2.0)
    psi0 = si.gaussian_guess(n, L, 77, vortex=True)
    _assert_ground_state_parity(*_solve_pair(n, L, par, psi0, trap={"kind": 0, "g": (1.0, 0.8)}))


def test_3d_ground_state_matches_oracle():
    n, L, par = (16, 16, 16), (5.0, 5.0, 5.0), (0.4, 0.5, 30.0, -1.0)
    trap = {"kind": 1, "g": (1.0, 1.0, 2.0), "quad": 0.0, "quart": 0.02}
    psi0 = si.gaussian_guess(n, L, 91)
    _assert_ground_state_parity(*_solve_pair(n, L, par, psi0, trap=trap))


def test_cascadic_multigrid_matches_oracle():
    n, L, par = (64, 64), (8.0, 8.0), (0.6, 0.3, 50.0, 0.5)
    models = [oracle_model((k, k), L, par) for k in (16, 32, 64)]
    psi0 = si.gaussian_guess((16, 16), L, 5, vortex=True)
    ref, levels = cm_pcg(models, psi0, Options(tol=1e-12, res_tol=1e-9))
    with Problem(n, L, [par]) as p:
        p.set_initial(psi0[None], level=2)
        res = p.solve(tol=1e-12, res_tol=1e-9, cm_levels=3)[0]
        got = p.psi()[0]
    assert res["total_iters"] > res["iters"]
    _assert_ground_state_parity(models[-1], ref, res, got)


def test_batch_results_equal_single_solves():
    # each solve of a batch gives the result it gives alone, within the parity tolerances
    # (tile shapes follow the total work, so the summation order may differ);
    # anisotropic trap: the minimisers are unique up to the global phase
    n, L = (32, 32), (6.0, 6.0)
    trap = {"kind": 0, "g": (1.0, 1.1)}
    pars = [(0.2, 0.4, 50.0, -2.0), (0.7, 1.1, 120.0, 3.0), (0.0, 0.0, 10.0, 0.0)]
    psis = np.stack([si.gaussian_guess(n, L, 200 + k) for k in range(3)])
    with Problem(n, L, pars, trap=trap) as p:
        p.set_initial(psis)
        rb = p.solve(tol=1e-12, res_tol=1e-9)
        gb = p.psi()
    for k in range(3):
        with Problem(n, L, [pars[k]], trap=trap) as p:
            p.set_initial(psis[k][None])
            r1 = p.solve(tol=1e-12, res_tol=1e-9)[0]
            g1 = p.psi()[0]
        assert rb[k]["status"] == "OK" and r1["status"] == "OK"
        assert rb[k]["energy"] == pytest.approx(r1["energy"], rel=1e-10)
        assert rb[k]["mu"] == pytest.approx(r1["mu"], rel=1e-10)
        assert np.max(np.abs(np.abs(gb[k]) ** 2 - np.abs(g1) ** 2)) < 1e-8


def test_status_codes():
    n, L = (32, 32), (6.0, 6.0)
    from paper_2602_17950_gb300 import GpsocError
    with Problem(n, L, [PAR]) as p:
        with pytest.raises(GpsocError, match="ESTATE"):
            p.solve()
        p.set_initial(si.gaussian_guess(n, L, 1)[None])
        r = p.solve(tol=1e-15, max_iter=3)[0]
        assert r["status"] == "ENOTCONV" and r["iters"] == 3
        with pytest.raises(GpsocError, match="EINVAL"):
            p.solve(tol=-1.0)
        with pytest.raises(GpsocError, match="EINVAL"):
            p.set_initial_kind([0, 1, 12])
    with pytest.raises(GpsocError, match="EINVAL"):
        Problem((12, 16), L, [PAR])


def test_nonfinite_input_is_reported():
    n, L = (32, 32), (6.0, 6.0)
    psi = si.gaussian_guess(n, L, 1)
    psi[0, 3, 3] = np.nan
    with Problem(n, L, [PAR]) as p:
        p.set_initial(psi[None])
        r = p.solve(tol=1e-12)[0]
    assert r["status"] == "ENONFINITE"


def test_mixed_precision_ground_state_matches_oracle():
    # FP32 transforms + FP64 reductions, then FP64 polishing: same tolerances as FP64.
    # An anisotropic trap removes the joint space-spin rotation symmetry of radial
    # traps, so the minimiser (and its density) is unique up to the global phase.
    n, L, par = (64, 64), (8.0, 8.0), (0.5, 0.5, 100.0, -1.0)
    trap = {"kind": 0, "g": (1.0, 1.15)}
    psi0 = si.gaussian_guess(n, L, si.seed_for(1, 0))
    m = oracle_model(n, L, par, trap)
    ref = pcg(m, psi0, Options(tol=1e-12, res_tol=2e-10))
    with Problem(n, L, [par], trap=trap) as p:
        p.set_initial(psi0[None])
        res = p.solve(tol=1e-12, res_tol=2e-10, precision=1, fp32_min_points=-1)[0]
        got = p.psi()[0]
    assert res["fp32_iters"] > 0 and res["fp64_iters"] > 0
    _assert_ground_state_parity(m, ref, res, got)


def test_mixed_precision_skips_fp32_on_small_levels():
    # MIXED keeps levels below fp32_min_points solve-points (default 65536) in FP64
    n, L, par = (64, 64), (8.0, 8.0), (0.5, 0.5, 100.0, -1.0)
    psi0 = si.gaussian_guess(n, L, si.seed_for(1, 0))
    with Problem(n, L, [par] * 4) as p:
        p.set_initial(np.stack([psi0] * 4))
        small = p.solve(tol=1e-10, precision=1, fp32_min_points=4 * 64 * 64 + 1)
        p.set_initial(np.stack([psi0] * 4))
        large = p.solve(tol=1e-10, precision=1, fp32_min_points=4 * 64 * 64)
    assert all(r["fp32_iters"] == 0 and r["status"] == "OK" for r in small)
    assert all(r["fp32_iters"] > 0 and r["status"] == "OK" for r in large)


def test_mixed_precision_radial_trap_invariants_match_oracle():
    # radial trap (config-1 parameters): the minimiser is degenerate under joint
    # spatial + spin rotation, so compare the invariant observables: E, mu, masses
    n, L, par = (64, 64), (8.0, 8.0), (0.5, 0.5, 100.0, -1.0)
    psi0 = si.gaussian_guess(n, L, si.seed_for(1, 0))
    m = oracle_model(n, L, par)
    ref = pcg(m, psi0, Options(tol=1e-12, res_tol=2e-10))
    with Problem(n, L, [par]) as p:
        p.set_initial(psi0[None])
        res = p.solve(tol=1e-12, res_tol=2e-10, precision=1, fp32_min_points=-1)[0]
    assert res["status"] == "OK"
    assert res["energy"] == pytest.approx(ref.energy, rel=1e-10)
    assert res["mu"] == pytest.approx(ref.mu, rel=1e-10)
    np.testing.assert_allclose(res["mass"], ref.masses, atol=1e-8)


def test_mixed_precision_cm_batch_matches_fp64():
    n, L = (64, 64), (8.0, 8.0)
    trap = {"kind": 0, "g": (1.0, 1.2)}
    pars = [(0.3, 0.7, 200.0, -3.0), (0.6, 0.2, 80.0, 5.0)]
    psis = np.stack([si.gaussian_guess((32, 32), L, 300 + k, vortex=True) for k in range(2)])
    out = {}
    for prec in (0, 1):
        with Problem(n, L, pars, trap=trap) as p:
            p.set_initial(psis, level=1)
            out[prec] = (p.solve(tol=1e-12, res_tol=2e-10, cm_levels=2, precision=prec, fp32_min_points=-1), p.psi())
    for k in range(2):
        r64, r32 = out[0][0][k], out[1][0][k]
        assert r64["status"] == "OK" and r32["status"] == "OK"
        assert r32["energy"] == pytest.approx(r64["energy"], rel=1e-10)
        assert r32["mu"] == pytest.approx(r64["mu"], rel=1e-10)
        assert np.max(np.abs(np.abs(out[1][1][k]) ** 2 - np.abs(out[0][1][k]) ** 2)) < 1e-8


@pytest.mark.parametrize("n,L", [((512, 512), (16.0, 16.0)), ((1024, 16), (20.0, 4.0)), ((16, 1024), (4.0, 20.0))])
def test_apply_h_large_tiles_match_oracle(n, L):
    # the largest tiles (384-thread blocks, radix-8 passes) in FP64
    psi = si.smooth_random_state(n, L, 51, width=min(L) / 3)[None]
    with Problem(n, L, [PAR]) as p:
        p.set_initial(psi)
        hp, obs = p.apply_h()
        phi = p.psi()[0]
    m = oracle_model(n, L, PAR)
    assert rel_max(hp[0], m.H(phi)) < 1e-11
    assert obs[0, 0] == pytest.approx(m.energy(phi), rel=1e-12)


@pytest.mark.parametrize("n", [64, 256, 512])
def test_fp32_iteration_kernels_run_at_every_tile_shape(n):
    # every kernel of the FP32 and FP64 iterations, at the tile shapes of each grid:
    # the profiled iterations run, the energy decreases and stays finite
    L = (16.0, 16.0)
    psi = si.gaussian_guess((n, n), L, 61, vortex=True)[None]
    with Problem((n, n), L, [(0.9, 1.0, 1000.0, -5.0)]) as p:
        for prec in (1, 0):
            p.set_initial(psi)
            E0 = p.observables()[0][0]
            prof = p.profile(iters=6, precision=prec)
            assert len(prof) == 9 and all(ms > 0 for _, ms in prof)
            E1, _, m = p.observables()
            assert np.isfinite(E1[0]) and E1[0] < E0
            assert abs(m[0].sum() - 1.0) < 1e-6


@pytest.mark.parametrize("precond", ["kinetic", "potential", "none"])
def test_preconditioner_variants_follow_oracle_step_by_step(precond):
    # P_Delta alone, P_V alone and no preconditioner (Section 3.4): 6 iterations from the
    # same input follow the oracle's iterations with the same preconditioner
    n, L = (64, 64), (8.0, 8.0)
    par = (0.5, 0.5, 100.0, -1.0)
    psi0 = si.gaussian_guess(n, L, si.seed_for(1, 0))
    m = oracle_model(n, L, par)
    ref = pcg(m, psi0, Options(tol=1e-300, max_iter=6, precond=precond))
    assert ref.iters == 6
    with Problem(n, L, [par]) as p:
        p.set_initial(psi0[None])
        res = p.iterate(6, precond=precond)[0]
        got = p.psi()[0]
    assert res["iters"] == 6
    assert rel_max(got, ref.Phi) < 1e-9
    assert res["energy"] == pytest.approx(ref.energies[-2], rel=1e-12)


@pytest.mark.parametrize("precond", ["kinetic", "potential"])
def test_preconditioner_variants_reach_the_oracle_ground_state(precond):
    # anisotropic trap: unique minimiser; each preconditioner reaches it (more
    # iterations than the combined one, as Section 3.4 reports)
    n, L, par = (32, 32), (6.0, 6.0), (0.4, 0.5, 40.0, -1.0)
    trap = {"kind": 0, "g": (1.0, 1.15)}
    psi0 = si.gaussian_guess(n, L, si.seed_for(1, 0))
    m = oracle_model(n, L, par, trap)
    ref = pcg(m, psi0, Options(tol=1e-12, res_tol=2e-10, precond=precond))
    with Problem(n, L, [par], trap=trap) as p:
        p.set_initial(psi0[None])
        res = p.solve(tol=1e-12, res_tol=2e-10, precond=precond)[0]
        got = p.psi()[0]
        p.set_initial(psi0[None])
        comb = p.solve(tol=1e-12, res_tol=2e-10)[0]
    _assert_ground_state_parity(m, ref, res, got)
    assert comb["energy"] == pytest.approx(res["energy"], rel=1e-10)
    assert comb["total_iters"] < res["total_iters"]


@pytest.mark.parametrize("omega", ["0.6", "0.7", "0.8", "0.9"])
def test_table_cpu_energies_on_the_gpu(omega):
    # Table table_cpu (Section 4, Example 3): the lowest energies printed to 4 decimals,
    # reached by CM-PCG 32 -> 64 -> 128 from guess (b) in every component, on the GPU
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "table_cpu.json")) as fh:
        gold = json.load(fh)
    par = (float(omega), 0.3, 50.0, 0.5)
    with Problem((128, 128), (12.0, 12.0), [par]) as p:
        p.set_initial_kind([1, 1, 1], level=2)
        res = p.solve(tol=1e-10, cm_levels=3, max_iter=200000)[0]
    assert res["status"] == "OK"
    assert abs(res["energy"] - gold["lowest_energy"][omega]) <= 0.5e-4


@pytest.mark.parametrize("stop,oracle_stop,tol", [(2, "residual", 1e-9), (1, "dphi", 1e-8)])
def test_stop_criteria_match_oracle(stop, oracle_stop, tol):
    # stop2 (max_l ||r_l||_inf < tol) and stop1 (max_l ||phi_l^n - phi_l^{n-1}||_inf < tol),
    # Section 3.4: the GPU stops where the oracle does (up to rounding at the threshold)
    # and its reported quantity satisfies the criterion
    n, L, par = (32, 32), (6.0, 6.0), (0.4, 0.5, 40.0, -1.0)
    trap = {"kind": 0, "g": (1.0, 1.15)}
    psi0 = si.gaussian_guess(n, L, si.seed_for(1, 0))
    m = oracle_model(n, L, par, trap)
    ref = pcg(m, psi0, Options(stop=oracle_stop, tol=tol))
    with Problem(n, L, [par], trap=trap) as p:
        p.set_initial(psi0[None])
        res = p.solve(stop=stop, tol=tol)[0]
    assert ref.status == "converged" and res["status"] == "OK"
    assert abs(res["iters"] - ref.iters) <= 2
    assert res["energy"] == pytest.approx(ref.energy, rel=1e-9)
    if stop == 2:
        assert res["res_inf"] < tol


_TRAP3 = {"kind": 1, "g": (1.0, 1.1, 2.0), "quad": 0.0, "quart": 0.02}


def test_3d_cascadic_multigrid_matches_oracle():
    # Algorithm 3 in 3D: 8^3 -> 16^3 by spectral zero padding, anisotropic harmonic-plus-quartic trap
    L, par = (5.0, 5.0, 5.0), (0.4, 0.5, 30.0, -1.0)
    models = [oracle_model((k, k, k), L, par, _TRAP3) for k in (8, 16)]
    psi0 = si.gaussian_guess((8, 8, 8), L, 93)
    ref, _ = cm_pcg(models, psi0, Options(tol=1e-12, res_tol=1e-9))
    with Problem((16, 16, 16), L, [par], trap=_TRAP3) as p:
        p.set_initial(psi0[None], level=1)
        res = p.solve(tol=1e-12, res_tol=1e-9, cm_levels=2)[0]
        got = p.psi()[0]
    assert res["levels"] == 2 and res["total_iters"] > res["iters"]
    _assert_ground_state_parity(models[-1], ref, res, got)


def test_3d_kinetic_preconditioner_follows_oracle_step_by_step():
    # the 3D preconditioner chain (y forward, z kinetic division, y inverse) with P_Delta alone
    n, L, par = (16, 16, 16), (5.0, 5.0, 5.0), (0.4, 0.5, 30.0, -1.0)
    psi0 = si.gaussian_guess(n, L, 94)
    m = oracle_model(n, L, par, _TRAP3)
    ref = pcg(m, psi0, Options(tol=1e-300, max_iter=6, precond="kinetic"))
    with Problem(n, L, [par], trap=_TRAP3) as p:
        p.set_initial(psi0[None])
        res = p.iterate(6, precond="kinetic")[0]
        got = p.psi()[0]
    assert res["iters"] == 6
    assert rel_max(got, ref.Phi) < 1e-9


def test_3d_mixed_precision_ground_state_matches_oracle():
    # FP32 phase forced on a small 3D grid, then FP64 polish: the oracle's FP64 ground state
    n, L, par = (16, 16, 16), (5.0, 5.0, 5.0), (0.4, 0.5, 30.0, -1.0)
    psi0 = si.gaussian_guess(n, L, 94)
    m = oracle_model(n, L, par, _TRAP3)
    ref = pcg(m, psi0, Options(tol=1e-12, res_tol=2e-10))
    with Problem(n, L, [par], trap=_TRAP3) as p:
        p.set_initial(psi0[None])
        res = p.solve(tol=1e-12, res_tol=2e-10, precision=1, fp32_min_points=-1)[0]
        got = p.psi()[0]
    assert res["fp32_iters"] > 0 and res["fp64_iters"] > 0
    _assert_ground_state_parity(m, ref, res, got)


def test_user_potential_ground_state_matches_oracle():
    # a user-supplied potential array on top of the harmonic trap, through every kernel that reads V
    n, L = (32, 32), (6.0, 6.0)
    X, Y = si.mesh(n, L)
    V = 0.3 * np.cos(X) * np.sin(0.5 * Y) + 0.1 * X
    trap = {"kind": 2, "g": (1.0, 1.15), "user_V": V}
    psi0 = si.gaussian_guess(n, L, 95)
    _assert_ground_state_parity(*_solve_pair(n, L, (0.3, 0.5, 40.0, -1.0), psi0, res_tol=2e-10, trap=trap))


def test_batched_parameters_match_individual_oracle_solves():
    # one batch, three parameter sets: each solve against its own oracle solve
    n, L = (32, 32), (6.0, 6.0)
    trap = {"kind": 0, "g": (1.0, 1.15)}
    pars = [(0.2, 0.3, 20.0, -1.0), (0.5, 1.0, 60.0, 2.0), (0.0, 0.0, 10.0, 0.0)]
    psi0 = [si.gaussian_guess(n, L, 96 + k) for k in range(3)]
    with Problem(n, L, pars, trap=trap) as p:
        p.set_initial(np.stack(psi0))
        res = p.solve(tol=1e-12, res_tol=2e-10)
        got = p.psi()
    for k in range(3):
        m = oracle_model(n, L, pars[k], trap)
        ref = pcg(m, psi0[k], Options(tol=1e-12, res_tol=2e-10))
        _assert_ground_state_parity(m, ref, res[k], got[k])
