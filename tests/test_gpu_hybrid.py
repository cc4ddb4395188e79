"""GPSOC_HYBRID against the FP64 oracle at the FP64 bars.

HYBRID keeps the wave function, H_lin Phi, the residual, every reduction of the
state and Algorithm 2 in FP64 and runs the preconditioner's and the search
direction's transforms in FP32; H_lin Phi is advanced by linearity and recomputed
exactly in FP64 every few iterations and before a residual is accepted.  Its
ground states must therefore meet the FP64 bars (E, mu to 1e-10 relative;
densities and component masses to 1e-8), and its first iterations follow the
oracle's to FP32 accuracy (the directions carry FP32 rounding)."""
import numpy as np
import pytest

import seeded_inputs as si
from oracle.model import Grid, Model
from oracle.pcg import Options, cm_pcg, pcg
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

HYBRID = 2


def _assert_parity(m, ref, res, got):
    assert ref.status == "converged" and res["status"] == "OK", res
    assert res["energy"] == pytest.approx(ref.energy, rel=1e-10)
    assert res["mu"] == pytest.approx(ref.mu, rel=1e-10)
    assert np.max(np.abs(np.abs(got) ** 2 - np.abs(ref.Phi) ** 2)) < 1e-8
    np.testing.assert_allclose(res["mass"], ref.masses, atol=1e-8)
    assert res["energy"] == pytest.approx(m.energy(got), rel=1e-12)   # observables of its own final state


@pytest.mark.parametrize("n,L,par,trap", [
    ((64, 64), (8.0, 8.0), (0.5, 0.5, 100.0, -1.0), {"kind": 0, "g": (1.0, 1.15)}),
    ((32, 64), (6.0, 10.0), (0.3, 0.9, 40.0, 2.0), {"kind": 0, "g": (1.0, 0.8)}),
    ((16, 16, 16), (5.0, 5.0, 5.0), (0.4, 0.5, 30.0, -1.0), {"kind": 1, "g": (1.0, 1.1, 2.0), "quad": 0.0,
                                                             "quart": 0.02}),
])
@pytest.mark.parametrize("lead", [0.0, -1.0])     # FP64 lead-in to max|r| < 1e-4, or none
def test_hybrid_ground_state_matches_oracle(n, L, par, trap, lead):
    psi0 = si.gaussian_guess(n, L, si.seed_for(1, 0), vortex=len(n) == 2)
    m = oracle_model(n, L, par, trap)
    ref = pcg(m, psi0, Options(tol=1e-12, res_tol=1e-9))
    with Problem(n, L, [par], trap=trap) as p:
        p.set_initial(psi0[None])
        res = p.solve(tol=1e-12, res_tol=1e-9, precision=HYBRID, hybrid_lead_res=lead)[0]
        got = p.psi()[0]
    assert res["fp32_iters"] > 0
    if lead < 0:
        assert res["fp64_iters"] == 0
    assert res["res_inf"] < 1e-9
    _assert_parity(m, ref, res, got)


def test_hybrid_iterations_follow_oracle():
    # the directions carry FP32 rounding, the state and every step decision FP64
    n, L, par = (64, 64), (8.0, 8.0), (0.5, 0.5, 100.0, -1.0)
    psi0 = si.gaussian_guess(n, L, si.seed_for(1, 0))
    m = oracle_model(n, L, par)
    ref = pcg(m, psi0, Options(tol=1e-300, max_iter=6))
    with Problem(n, L, [par]) as p:
        p.set_initial(psi0[None])
        res = p.iterate(6, precision=HYBRID)[0]
        got = p.psi()[0]
    assert res["iters"] == 6
    assert rel_max(got, ref.Phi) < 1e-4
    assert res["energy"] == pytest.approx(ref.energies[-2], rel=1e-6)
    assert abs(m.mass(got) - 1.0) < 1e-13           # the update keeps the FP64 normalisation


def test_hybrid_cascadic_multigrid_batch_matches_oracle():
    n, L = (64, 64), (8.0, 8.0)
    trap = {"kind": 0, "g": (1.0, 1.2)}
    pars = [(0.3, 0.7, 200.0, -3.0), (0.6, 0.2, 80.0, 5.0)]
    psis = np.stack([si.gaussian_guess((32, 32), L, 300 + k, vortex=True) for k in range(2)])
    with Problem(n, L, pars, trap=trap) as p:
        p.set_initial(psis, level=1)
        res = p.solve(tol=1e-12, res_tol=1e-9, cm_levels=2, precision=HYBRID)
        got = p.psi()
    for k in range(2):
        models = [oracle_model((j, j), L, pars[k], trap) for j in (32, 64)]
        ref, _ = cm_pcg(models, psis[k], Options(tol=1e-12, res_tol=1e-9))
        _assert_parity(models[-1], ref, res[k], got[k])


def test_hybrid_served_results_equal_solving_alone():
    from paper_2602_17950_gb300 import Server
    trap = {"kind": 0, "g": (1.0, 1.1, 1.2)}
    reqs = [((32, 32), (6.0, 6.0), (0.3, 0.5, 60.0, -1.0)), ((64, 64), (8.0, 8.0), (0.5, 0.8, 100.0, 2.0)),
            ((16, 16, 16), (5.0, 5.0, 5.0), (0.2, 0.4, 30.0, -2.0)), ((32, 32), (6.0, 6.0), (0.0, 1.2, 20.0, 0.0))]
    # mu moves to first order with the state: requests with soft modes need a tight residual
    opts = dict(tol=1e-13, res_tol=5e-11)
    guesses = [si.gaussian_guess(n, L, 410 + k, vortex=(len(n) == 2)) for k, (n, L, _) in enumerate(reqs)]
    done = {}
    with Server(hbm_budget_bytes=8e9, slots_per_bucket=4, precision=HYBRID, iters_per_step=16) as sv:
        tickets = [sv.submit(n, L, par, guesses[k], trap=trap, **opts) for k, (n, L, par) in enumerate(reqs)]
        for k, t in enumerate(tickets):
            got = sv.poll(t, timeout_ms=-1)
            assert got is not None
            done[k] = got
    for k, (n, L, par) in enumerate(reqs):
        r, psi = done[k]
        with Problem(n, L, [par], trap=trap) as p:
            p.set_initial(guesses[k][None])
            ra = p.solve(**opts)[0]
            pa = p.psi()[0]
        assert r["status"] == "OK" and ra["status"] == "OK", (k, r, ra)
        assert r["res_inf"] < 5e-11
        assert r["energy"] == pytest.approx(ra["energy"], rel=1e-10)
        assert r["mu"] == pytest.approx(ra["mu"], rel=1e-10)
        assert np.max(np.abs(np.abs(psi) ** 2 - np.abs(pa) ** 2)) < 1e-8
