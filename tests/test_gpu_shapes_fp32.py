"""GPU parity of the FP32 kernels and of the multi-line tile shapes, against the FP64 oracle.

FP32 bars (the arrays are FP32, every block and grid sum and every scalar FP64):
operator outputs within 1e-5 of the oracle's max magnitude (FP32 rounding of
a few transforms of log2(n) <= 10 passes each, eps_32 = 6e-8); reduced
scalars (E, mu, alpha_l, masses) within 1e-6 relative, a_n (a difference
-mu + <H P, P>/|P|^2) at the array bar, and b_n, a sum
with cancellation that projects the error of H Phi, within the array bar times
the size of its terms (2 ||H Phi||).  FP64 bars
as in test_gpu_parity.py (1e-11 of the max magnitude, 1e-12 relative).

The tile shapes follow the total work (lines per tile grow with the batch:
rows R per x tile, columns TC per y/z tile); the cases below reach R in
{2, 4, 8, 16} and TC in {4, 8, 16, 32}, the shapes of the batched workloads, and
each case asserts the shape it runs.  Algorithm 2's branches (the theta_trial
step for a <= 0, backtracking halvings, the Step 2 -> Step 1 restart with
beta = 0) are followed step by step on a trajectory that takes all of them."""
import math

import numpy as np
import pytest

import seeded_inputs as si
from oracle.model import Model
from oracle.pcg import Options, pcg
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

FP64, FP32 = 0, 1
BARS = {FP64: dict(arr=1e-11, scal=1e-12), FP32: dict(arr=1e-5, scal=1e-6)}
TRAP = {"kind": 1, "g": (1.0, 1.3, 0.7), "quad": -0.1, "quart": 0.02}

# (grid, box, batch, expected lines per tile along x, y[, z])
SHAPES = [
    ((64, 64), (8.0, 8.0), 64, (8, 8)),
    ((64, 64), (8.0, 8.0), 128, (8, 16)),
    ((128, 128), (10.0, 10.0), 16, (4, 4)),
    ((256, 256), (12.0, 12.0), 8, (2, 4)),
    ((32, 32), (6.0, 6.0), 40, (4, 4)),
    ((64, 64, 64), (7.0, 7.0, 7.0), 4, (8, 16, 16)),
    ((32, 32, 128), (6.0, 6.0, 9.0), 4, (16, 32, 8)),
]


def _params(batch, seed):
    return [(q.Omega, q.gamma, q.beta0, q.beta1) for q in si.batch_params(seed, batch)]


def _states(n, L, batch, seed):
    return np.stack([si.smooth_random_state(n, L, seed + k, width=min(L) / 3) for k in range(batch)])


def _assert_shape(p, n, expect):
    for axis, lines in enumerate(expect):
        for prec in (FP64, FP32):
            assert p.tile_shape(axis, precision=prec)[0] == lines, (axis, prec)


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("n,L,batch,expect", SHAPES)
def test_apply_h_at_batched_tile_shapes_matches_oracle(n, L, batch, expect, prec):
    pars = _params(batch, 7000 + batch)
    psi = _states(n, L, batch, 100)
    with Problem(n, L, pars, trap=TRAP) as p:
        _assert_shape(p, n, expect)
        p.set_initial(psi)
        hp, obs = p.apply_h(precision=prec)
        phi = p.psi()
    bar = BARS[prec]
    for k in range(0, batch, max(1, batch // 8)):     # every solve's own parameters; a spread of slots
        m = oracle_model(n, L, pars[k], TRAP)
        H = m.H(phi[k])
        assert rel_max(hp[k], H) < bar["arr"], k
        assert obs[k, 0] == pytest.approx(m.energy(phi[k]), rel=bar["scal"])
        assert obs[k, 1] == pytest.approx(m.mu(phi[k], H), rel=bar["scal"])
        np.testing.assert_allclose(obs[k, 2:5], m.alpha(phi[k]), rtol=bar["scal"])
        np.testing.assert_allclose(obs[k, 5:8], m.masses(phi[k]), rtol=bar["scal"], atol=1e-15)


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("n,L,batch,expect", [SHAPES[0], SHAPES[2], SHAPES[5], SHAPES[6]])
def test_preconditioner_and_step_model_at_batched_tile_shapes_match_oracle(n, L, batch, expect, prec):
    pars = _params(batch, 7100 + batch)
    psi = _states(n, L, batch, 300)
    r = np.stack([si.random_state(n, 400 + k) for k in range(batch)])
    D = _states(n, L, batch, 500)
    thetas = np.array([0.9, 0.2, 1e-3])
    with Problem(n, L, pars, trap=TRAP) as p:
        _assert_shape(p, n, expect)
        p.set_initial(psi)
        phi = p.psi()
        z = p.apply_precond(r, precision=prec)
        models = [oracle_model(n, L, par, TRAP) for par in pars]
        P = np.stack([D[k] - models[k].inner(D[k], phi[k]).real * phi[k] for k in range(batch)])
        out = p.step_model(P, thetas, precision=prec)
    bar = BARS[prec]
    for k in range(0, batch, max(1, batch // 4)):
        m = models[k]
        assert rel_max(z[k], m.precond_C(r[k], phi[k], m.alpha(phi[k]))) < bar["arr"], k
        H = m.H(phi[k])
        a, b = m.step_coefficients(phi[k], P[k], H, m.mu(phi[k], H))
        assert out[k, 0] == pytest.approx(a, rel=bar["arr"])   # a_n = -mu + <H P, P>/|P|^2: a difference
        # b_n = 2 Re<H Phi, P>/||P|| sums terms of size |H Phi||P| to a residual-sized result (P is
        # tangent): it carries the error of H Phi, so its bar is the array bar times 2 ||H Phi||
        assert out[k, 1] == pytest.approx(b, rel=bar["scal"], abs=bar["arr"] * 2 * math.sqrt(m.mass(H)))
        Ph = P[k] / math.sqrt(m.mass(P[k]))
        E = abs(m.energy(phi[k]))
        for j, t in enumerate(thetas):
            ref = m.energy_change(phi[k], Ph, t)
            assert out[k, 2 + j] == pytest.approx(ref, rel=10 * bar["scal"], abs=bar["scal"] * E * abs(t)), (k, t)


@pytest.mark.parametrize("n,L", [((64, 64), (8.0, 8.0)), ((32, 64), (6.0, 9.0)), ((16, 16, 32), (4.0, 4.0, 5.0))])
def test_fp32_operators_match_oracle_single_solve(n, L):
    par = (0.45, 0.8, 30.0, -4.0)
    psi = si.smooth_random_state(n, L, 61, width=min(L) / 3)[None]
    r = si.random_state(n, 62)[None]
    with Problem(n, L, [par], trap=TRAP) as p:
        p.set_initial(psi)
        hp, obs = p.apply_h(precision=FP32)
        z = p.apply_precond(r, precision=FP32)
        phi = p.psi()[0]
    m = oracle_model(n, L, par, TRAP)
    H = m.H(phi)
    assert rel_max(hp[0], H) < 1e-5
    assert obs[0, 8] == pytest.approx(m.inner(m.H_lin(phi), phi).real, rel=1e-6)
    assert rel_max(z[0], m.precond_C(r[0], phi, m.alpha(phi))) < 1e-5


def test_fp32_iterations_follow_oracle_trajectory():
    # N FP32 PCG iterations (FP64 sums and step decisions) against the oracle's first N FP64
    # iterations from the same input: the trajectories agree to FP32 accuracy
    n, L, par = (64, 64), (8.0, 8.0), (0.5, 0.5, 100.0, -1.0)
    psi0 = si.gaussian_guess(n, L, si.seed_for(1, 0))
    m = oracle_model(n, L, par)
    ref = pcg(m, psi0, Options(tol=1e-300, max_iter=6))
    with Problem(n, L, [par]) as p:
        p.set_initial(psi0[None])
        res = p.iterate(6, precision=FP32)[0]
        got = p.psi()[0]
    assert res["iters"] == 6 and res["fp32_iters"] == 6
    assert rel_max(got, ref.Phi) < 1e-4
    assert res["energy"] == pytest.approx(ref.energies[-2], rel=1e-6)


@pytest.mark.parametrize("prec,bar", [(FP64, 1e-9), (FP32, 1e-4)])
def test_batched_iterations_at_large_tiles_follow_oracle(prec, bar):
    # 64 solves of 64^2 (R = 8 rows per x tile, TC = 8 columns per y tile): every kernel of
    # the iteration at the tile shape of the batched workloads, against the oracle per solve
    n, L, batch = (64, 64), (8.0, 8.0), 64
    pars = _params(batch, 7200)
    psi0 = np.stack([si.gaussian_guess(n, L, 900 + k, vortex=bool(k % 2)) for k in range(batch)])
    with Problem(n, L, pars) as p:
        _assert_shape(p, n, (8, 8))
        p.set_initial(psi0)
        res = p.iterate(4, precision=prec)
        got = p.psi()
    for k in range(0, batch, 9):
        m = oracle_model(n, L, pars[k])
        ref = pcg(m, psi0[k], Options(tol=1e-300, max_iter=4))
        assert res[k]["iters"] == 4 == ref.iters
        assert rel_max(got[k], ref.Phi) < bar, k


def test_algorithm2_branches_follow_oracle():
    # a trajectory that takes the theta_trial step (a_n <= 0), backtracking halvings and a
    # Step 2 -> Step 1 restart with beta = 0 (Algorithm 2): the GPU takes the same branches
    # (same halving and restart counts) and the same iterates as the oracle
    n, L = (32, 32), (6.0, 6.0)
    trap = {"kind": 0, "g": (1.0, 1.1)}
    par = (0.95, 2.0, 2000.0, -10.0)
    psi0 = si.gaussian_guess(n, L, 501, vortex=True)
    m = oracle_model(n, L, par, trap)
    seen = []
    orig = Model.step_coefficients

    def record(self, Phi, P, HPhi, mu):
        a, b = orig(self, Phi, P, HPhi, mu)
        seen.append((a, b))
        return a, b
    Model.step_coefficients = record
    try:
        ref = pcg(m, psi0, Options(tol=1e-300, max_iter=10))
    finally:
        Model.step_coefficients = orig
    assert ref.iters == 10 and ref.beta_resets >= 1 and ref.halvings >= 3
    assert any(a <= 0 and b < 0 for a, b in seen)          # the theta_trial branch was taken
    with Problem(n, L, [par], trap=trap) as p:
        p.set_initial(psi0[None])
        res = p.iterate(10)[0]
        got = p.psi()[0]
    assert res["iters"] == 10
    assert res["halvings"] == ref.halvings
    assert res["beta_resets"] == ref.beta_resets
    assert rel_max(got, ref.Phi) < 1e-9
    # E of an iterate away from the minimum moves to first order with the iterate (bar 1e-9);
    # with c0 = 2000 the rounding of ten stiff steps reaches about 2e-12 of E, while a
    # different branch would change E by a whole step's energy change
    assert res["energy"] == pytest.approx(ref.energies[-2], rel=1e-11)
