"""Every tile the autotuner can choose, against the FP64 oracle.

The tile of the passes along an axis (lines per block, FFT elements per thread)
is chosen per grid, batch and kernel precision, by the built-in rule or by
gpsoc_autotune.  Here every valid candidate of every axis is set in turn and
the operators (H(Phi) with its observables, P_C r, the step model) are compared
with the oracle at the bars of the other operator tests: FP64 kernels 1e-11 of
the max magnitude and 1e-12 relative for reduced scalars; FP32 kernels 1e-5 and
1e-6, with a_n (a difference -mu + <H P, P>/|P|^2) at the array bar and b_n (a sum
with cancellation that projects the error of H Phi) at the array bar times the
size of its terms.  Then an
autotuned problem solves to the oracle's ground state."""
import math

import numpy as np
import pytest

import seeded_inputs as si
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
PARS = [(0.45, 0.8, 30.0, -4.0), (0.9, 0.2, 120.0, 2.0)]


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("n,L", [((32, 64), (6.0, 9.0)), ((16, 16, 32), (4.0, 4.0, 5.0))])
def test_every_tile_candidate_matches_oracle(n, L, prec):
    pars = PARS[:2] if len(n) == 2 else PARS[:1]
    B = len(pars)
    psi = np.stack([si.smooth_random_state(n, L, 80 + k, width=min(L) / 3) for k in range(B)])
    r = np.stack([si.random_state(n, 90 + k) for k in range(B)])
    D = np.stack([si.smooth_random_state(n, L, 95 + k, width=min(L) / 3) for k in range(B)])
    thetas = np.array([0.7, 1e-2])
    bar = BARS[prec]
    with Problem(n, L, pars, trap=TRAP) as p:
        p.set_initial(psi)
        phi = p.psi()
        models = [oracle_model(n, L, par, TRAP) for par in pars]
        ref = []
        for k, m in enumerate(models):
            H = m.H(phi[k])
            P = D[k] - m.inner(D[k], phi[k]).real * phi[k]
            a, b = m.step_coefficients(phi[k], P, H, m.mu(phi[k], H))
            Ph = P / math.sqrt(m.mass(P))
            ref.append(dict(H=H, E=m.energy(phi[k]), z=m.precond_C(r[k], phi[k], m.alpha(phi[k])), P=P, a=a, b=b,
                            dE=[m.energy_change(phi[k], Ph, t) for t in thetas], Hn=math.sqrt(m.mass(H))))
        Ps = np.stack([x["P"] for x in ref])
        tried = 0
        try:
            for axis in range(len(n)):
                for lines, ept in p.tile_candidates(axis, precision=prec):
                    p.tuning_set(axis, lines, ept, precision=prec)
                    assert p.tile_shape(axis, precision=prec)[:2] == (lines, ept)
                    hp, obs = p.apply_h(precision=prec)
                    z = p.apply_precond(r, precision=prec)
                    out = p.step_model(Ps, thetas, precision=prec)
                    for k in range(B):
                        x = ref[k]
                        tag = (axis, lines, ept, k)
                        assert rel_max(hp[k], x["H"]) < bar["arr"], tag
                        assert obs[k, 0] == pytest.approx(x["E"], rel=bar["scal"]), tag
                        assert rel_max(z[k], x["z"]) < bar["arr"], tag
                        assert out[k, 0] == pytest.approx(x["a"], rel=bar["arr"]), tag   # -mu + <H P, P>/|P|^2
                        assert out[k, 1] == pytest.approx(x["b"], rel=bar["scal"], abs=bar["arr"] * 2 * x["Hn"]), tag
                        E = abs(x["E"])
                        for j, t in enumerate(thetas):
                            assert out[k, 2 + j] == pytest.approx(x["dE"][j], rel=10 * bar["scal"],
                                                                  abs=bar["scal"] * E * t), tag
                    tried += 1
                p.tuning_set(axis, 0, 0, precision=prec)
        finally:
            for axis in range(len(n)):
                p.tuning_set(axis, 0, 0, precision=prec)
    assert tried >= 20


@pytest.mark.parametrize("prec", [FP64, 2])
def test_autotuned_tiles_solve_to_the_oracle_ground_state(prec):
    n, L = (64, 64), (8.0, 8.0)
    trap = {"kind": 0, "g": (1.0, 1.15)}
    pars = [(0.5, 0.5, 100.0, -1.0), (0.3, 0.9, 60.0, 2.0), (0.0, 0.4, 40.0, -1.0)]
    psi0 = [si.gaussian_guess(n, L, 500 + k) for k in range(3)]
    with Problem(n, L, pars, trap=trap) as p:
        try:
            p.set_initial(np.stack(psi0))
            chosen = p.autotune(iters=4, precision=prec)
            kp = FP64 if prec == FP64 else FP32
            for axis, tile in enumerate(chosen):
                assert tile == p.tile_shape(axis, precision=kp)[:2]
                assert tile in p.tile_candidates(axis, precision=kp) or tile[0] > 0
            p.set_initial(np.stack(psi0))
            res = p.solve(tol=1e-12, res_tol=2e-10, precision=prec)
            got = p.psi()
        finally:
            for axis in range(2):
                p.tuning_set(axis, 0, 0, precision=FP64 if prec == FP64 else FP32)
    for k in range(3):
        m = oracle_model(n, L, pars[k], trap)
        ref = pcg(m, psi0[k], Options(tol=1e-12, res_tol=2e-10))
        assert res[k]["status"] == "OK" and ref.status == "converged"
        assert res[k]["energy"] == pytest.approx(ref.energy, rel=1e-10)
        assert np.max(np.abs(np.abs(got[k]) ** 2 - np.abs(ref.Phi) ** 2)) < 1e-8
