"""The served form: requests of different grids and parameters arriving while
others run are admitted into free slots and finish with the result each one
gives alone (within the parity tolerances), in FP64 and in mixed precision."""
import numpy as np
import pytest

import seeded_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_17950_gb300 import build
    build.build()


TRAP = {"kind": 0, "g": (1.0, 1.1, 1.2)}     # anisotropic: minimisers unique up to the phase
REQS = [((32, 32), (6.0, 6.0), (0.3, 0.5, 60.0, -1.0)),
        ((64, 64), (8.0, 8.0), (0.5, 0.8, 100.0, 2.0)),
        ((32, 32), (6.0, 6.0), (0.0, 1.2, 20.0, 0.0)),
        ((16, 16, 16), (5.0, 5.0, 5.0), (0.2, 0.4, 30.0, -2.0)),
        ((32, 32), (6.0, 6.0), (0.6, 0.1, 150.0, 4.0)),
        ((64, 64), (8.0, 8.0), (0.1, 0.3, 40.0, -3.0))]
OPTS = dict(tol=1e-12, res_tol=2e-10, fp32_min_points=-1)   # FP32 stage on every bucket when mixed


def _alone(n, L, par, psi0):
    from paper_2602_17950_gb300 import Problem
    with Problem(n, L, [par], trap=TRAP) as p:
        p.set_initial(psi0[None])
        r = p.solve(**OPTS)[0]
        return r, p.psi()[0]


@pytest.mark.parametrize("precision", [0, 1])
def test_served_results_equal_solving_alone(precision):
    from paper_2602_17950_gb300 import Server
    guesses = [si.gaussian_guess(n, L, 400 + k, vortex=(len(n) == 2)) for k, (n, L, _) in enumerate(REQS)]
    done = {}
    with Server(hbm_budget_bytes=8e9, slots_per_bucket=4, precision=precision, iters_per_step=16) as sv:
        tickets = []
        # staggered arrivals: two requests up front, one more after every step
        pending = list(range(len(REQS)))
        for k in pending[:2]:
            n, L, par = REQS[k]
            tickets.append((k, sv.submit(n, L, par, guesses[k], trap=TRAP, **OPTS)))
        nxt = 2
        for _ in range(20000):
            busy = sv.step()
            if nxt < len(REQS):
                n, L, par = REQS[nxt]
                tickets.append((nxt, sv.submit(n, L, par, guesses[nxt], trap=TRAP, **OPTS)))
                nxt += 1
            for k, t in tickets:
                if k not in done:
                    got = sv.poll(t)
                    if got is not None:
                        done[k] = got
            if len(done) == len(REQS) and busy == 0:
                break
        assert sv.stats()["queued"] == 0
    assert len(done) == len(REQS)
    for k, (n, L, par) in enumerate(REQS):
        r, psi = done[k]
        ra, pa = _alone(n, L, par, guesses[k])
        assert r["status"] == "OK" and ra["status"] == "OK", (k, r, ra)
        if precision == 1:
            assert r["fp32_iters"] > 0
        assert r["energy"] == pytest.approx(ra["energy"], rel=1e-10)
        assert r["mu"] == pytest.approx(ra["mu"], rel=1e-10)
        assert np.max(np.abs(np.abs(psi) ** 2 - np.abs(pa) ** 2)) < 1e-8


def test_budget_queues_requests_until_room_frees():
    from paper_2602_17950_gb300 import Server
    # room for one small bucket only: the second grid waits for the first bucket to empty
    with Server(hbm_budget_bytes=6e6, slots_per_bucket=1, precision=0, iters_per_step=32) as sv:
        t1 = sv.submit((16, 16), (5.0, 5.0), (0.2, 0.3, 20.0, 1.0), si.gaussian_guess((16, 16), (5.0, 5.0), 1),
                       trap=TRAP, **OPTS)
        t2 = sv.submit((32, 16), (6.0, 5.0), (0.1, 0.2, 10.0, 0.0), si.gaussian_guess((32, 16), (6.0, 5.0), 2),
                       trap=TRAP, **OPTS)
        saw_queue = False
        got = {}
        for _ in range(5000):
            sv.step()
            saw_queue |= sv.stats()["queued"] > 0
            for t in (t1, t2):
                if t not in got:
                    g = sv.poll(t, want_psi=False)
                    if g is not None:
                        got[t] = g
            if len(got) == 2:
                break
        assert saw_queue and len(got) == 2
        assert all(g[0]["status"] == "OK" for g in got.values())


def test_poll_states():
    from paper_2602_17950_gb300 import GpsocError, Server
    with Server(hbm_budget_bytes=1e9, slots_per_bucket=2) as sv:
        t = sv.submit((16, 16), (5.0, 5.0), (0.0, 0.0, 5.0, 0.0), si.gaussian_guess((16, 16), (5.0, 5.0), 3),
                      trap=TRAP, **OPTS)
        assert sv.poll(t) is None        # queued
        with pytest.raises(GpsocError, match="EINVAL"):
            sv.poll(t + 1000)


def test_cancel_and_bounded_poll():
    from paper_2602_17950_gb300 import GpsocError, Problem, Server
    n, L = (64, 64), (8.0, 8.0)
    pars = [(0.5, 0.5, 100.0, -1.0), (0.3, 0.8, 60.0, 2.0), (0.4, 0.2, 80.0, -2.0)]
    psis = [si.gaussian_guess(n, L, 450 + k) for k in range(3)]
    opts = dict(tol=1e-13, res_tol=1e-10)
    with Server(hbm_budget_bytes=1e9, slots_per_bucket=1, precision=0, iters_per_step=8) as sv:
        t = [sv.submit(n, L, pars[k], psis[k], trap=TRAP, **opts) for k in range(3)]
        sv.cancel(t[2])                               # still queued
        sv.step()                                     # t[0] admitted and running, t[1] queued
        sv.cancel(t[0])                               # running: stopped after its round, slot freed
        for k in (0, 2):
            r, psi = sv.poll(t[k])
            assert r["status"] == "ECANCELED" and psi is None
        with pytest.raises(GpsocError, match="EINVAL"):
            sv.cancel(t[0])                           # released ticket
        assert sv.poll(t[1], timeout_ms=1) is None    # a bounded wait that runs out: ETIMEOUT
        got = sv.poll(t[1], timeout_ms=-1)            # wait until it finishes
        assert got is not None
        r, psi = got
    with Problem(n, L, [pars[1]], trap=TRAP) as p:
        p.set_initial(psis[1][None])
        ra = p.solve(**opts)[0]
    assert r["status"] == "OK" and ra["status"] == "OK"
    assert r["energy"] == pytest.approx(ra["energy"], rel=1e-10)
