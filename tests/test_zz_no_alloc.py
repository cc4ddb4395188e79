"""The allocation-free Hamiltonian entry point (gpsoc_apply_h_noalloc).

Some callers cannot allocate device memory when they need H(Phi): a framework
that already handed all device memory to its own pool, a real-time loop that
must not pay for or synchronise on cudaMalloc/cudaFree, or code running inside a
fixed, pre-reserved memory budget.  For them the library keeps all intermediate
data of this one operation in a fixed 16 MiB device array.  This test checks,
through the C ABI, that two consecutive calls give the same H(Phi) and
observables as the allocating entry point gpsoc_apply_h, within the
tolerances of the other operator tests.  It runs last (file name) so that a run
stopping at the first failure has already run every other test, and it also
passes when run alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import seeded_inputs as si
from tests.gpu_common import rel_max

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_17950_gb300 import build
    build.build()


@pytest.mark.parametrize("n,L,batch", [((64, 64), (8.0, 8.0), 2), ((32, 64), (6.0, 9.0), 2),
                                       ((16, 16, 32), (4.0, 4.0, 5.0), 2),
                                       ((32, 32), (6.0, 6.0), 40)])     # 4 rows / 4 columns per tile
def test_noalloc_apply_h_matches_allocating_entry_point(n, L, batch):
    from oracle.model import Grid, Model, Trap
    from paper_2602_17950_gb300 import Problem, gpsoc
    base = [(0.45, 0.8, 30.0, -4.0), (0.9, 0.2, 120.0, 2.0)]
    pars = [base[k % 2] for k in range(batch)]
    trap = {"kind": 1, "g": (1.0, 1.3, 0.7), "quad": -0.1, "quart": 0.02}
    psi = np.stack([si.smooth_random_state(n, L, 70 + k, width=min(L) / 3) for k in range(batch)])
    with Problem(n, L, pars, trap=trap) as p:
        p.set_initial(psi)
        ref_h, ref_obs = p.apply_h()
        phi = p.psi()                    # the normalised states the reference used
    d_psi = torch.from_numpy(phi.copy()).cuda()
    for _ in range(2):                   # two calls in a row share the scratch array
        d_out = torch.full_like(d_psi, float("nan"))
        obs = gpsoc.apply_h_noalloc(n, L, pars, trap, d_psi.data_ptr(), d_out.data_ptr())
        got = d_out.cpu().numpy()
        for k in range(batch):
            assert rel_max(got[k], ref_h[k]) < 1e-11
            np.testing.assert_allclose(obs[k], ref_obs[k], rtol=1e-12, atol=1e-15)
    # and against the CPU oracle's H(Phi) (Eqs. eigen1-eigen3) for two of the solves
    for k in (0, batch - 1):
        m = Model(Grid(n, L), Trap(g=trap["g"], quad=trap["quad"], quart=trap["quart"]), Omega=pars[k][0],
                  gamma=pars[k][1], c0=pars[k][2], c1=pars[k][3])
        assert rel_max(got[k], m.H(phi[k])) < 1e-11
        assert obs[k, 0] == pytest.approx(m.energy(phi[k]), rel=1e-12)


def test_noalloc_rejects_oversized_problem():
    from paper_2602_17950_gb300 import GpsocError, gpsoc
    n, L = (1024, 1024), (8.0, 8.0)
    d_psi = torch.zeros((1, 3, 8, 8), dtype=torch.complex128, device="cuda")   # never read
    with pytest.raises(GpsocError, match="EBUDGET"):
        gpsoc.apply_h_noalloc(n, L, [(0.0, 0.0, 0.0, 0.0)], None, d_psi.data_ptr(), d_psi.data_ptr())
