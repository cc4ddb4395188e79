"""The exact step size of Eq. theta on the GPU against the oracle.

theta_n = argmin_{theta > 0} E(cos(theta) Phi + sin(theta) P/|P|) is found on both sides
on the explicit sin/cos form of E(theta) (Section 3.1): the GPU by Newton steps on the
reduced integrals, the oracle by Brent's root finder on its own integrals.  Both
reach the same minimiser to rounding, so the iterations agree as tightly as with
Algorithm 2's quadratic model (Phi to 1e-9 of its max, E to 1e-12), and the
ground states meet the FP64 bars."""
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


@pytest.mark.parametrize("n,L,par", [((64, 64), (8.0, 8.0), (0.5, 0.5, 100.0, -1.0)),
                                     ((16, 16, 16), (5.0, 5.0, 5.0), (0.4, 0.5, 30.0, -1.0))])
def test_exact_step_follows_oracle_step_by_step(n, L, par):
    psi0 = si.gaussian_guess(n, L, si.seed_for(1, 0))
    m = oracle_model(n, L, par)
    ref = pcg(m, psi0, Options(tol=1e-300, max_iter=6, line_search="exact"))
    assert ref.iters == 6
    with Problem(n, L, [par]) as p:
        p.set_initial(psi0[None])
        res = p.iterate(6, line_search="exact")[0]
        got = p.psi()[0]
    assert res["iters"] == 6
    assert rel_max(got, ref.Phi) < 1e-9
    assert res["energy"] == pytest.approx(ref.energies[-2], rel=1e-12)


@pytest.mark.parametrize("n,L,par", [((16, 16), (5.0, 5.0), (0.3, 0.5, 20.0, -1.0)),
                                     ((32, 32), (6.0, 6.0), (0.2, 0.4, 10.0, 1.0))])
def test_exact_step_ground_state_matches_oracle(n, L, par):
    trap = {"kind": 0, "g": (1.0, 1.15)}
    psi0 = si.gaussian_guess(n, L, 7)
    m = oracle_model(n, L, par, trap)
    ref = pcg(m, psi0, Options(tol=1e-12, res_tol=1e-9, line_search="exact"))
    with Problem(n, L, [par], trap=trap) as p:
        p.set_initial(psi0[None])
        res = p.solve(tol=1e-12, res_tol=1e-9, line_search="exact")[0]
        got = p.psi()[0]
    assert ref.status == "converged" and res["status"] == "OK"
    assert abs(res["iters"] - ref.iters) <= 2
    assert res["energy"] == pytest.approx(ref.energy, rel=1e-10)
    assert res["mu"] == pytest.approx(ref.mu, rel=1e-10)
    assert np.max(np.abs(np.abs(got) ** 2 - np.abs(ref.Phi) ** 2)) < 1e-8
