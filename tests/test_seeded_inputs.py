"""The seeded input generators shared by the oracle side and the GPU side: they are
deterministic, follow their stated distributions and normalisation, and hold none of
the method's arithmetic."""
import math

import numpy as np

import seeded_inputs as si


def test_splitmix64_reference_values():
    # SplitMix64 from seed 0: the first outputs of the published generator
    r = si.SplitMix64(0)
    assert [r.next() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_gaussian_guess_is_deterministic_and_normalised_per_component():
    n, L = (32, 48), (6.0, 8.0)
    a = si.gaussian_guess(n, L, 1234)
    b = si.gaussian_guess(n, L, 1234)
    assert a.shape == (3, 48, 32) and np.array_equal(a, b)
    dV = (2 * L[0] / n[0]) * (2 * L[1] / n[1])
    for c in range(3):
        assert math.isclose(dV * np.sum(np.abs(a[c]) ** 2), 1.0 / 3.0, rel_tol=1e-12)
    assert not np.array_equal(a, si.gaussian_guess(n, L, 1235))


def test_batch_params_ranges():
    ps = si.batch_params(si.seed_for(3, 0), 500)
    om = np.array([p.Omega for p in ps]); ga = np.array([p.gamma for p in ps])
    b0 = np.array([p.beta0 for p in ps]); b1 = np.array([p.beta1 for p in ps])
    assert om.min() >= 0 and om.max() < 0.95 and ga.min() >= 0 and ga.max() < 2
    assert b0.min() >= 100 and b0.max() < 2000 and b1.min() >= -10 and b1.max() < 10
    assert abs(om.mean() - 0.475) < 0.05 and abs(b1.mean()) < 1.0


def test_serve_trace_is_poisson_and_uses_every_grid():
    rate = 4.0
    tr = si.serve_trace(si.seed_for(5, 0), 2000, rate)
    t = np.array([q["arrival"] for q in tr])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1 / rate) < 0.05 / rate * 4            # exponential gaps, mean 1/rate
    assert abs(gaps.std() - 1 / rate) < 0.1 / rate * 4
    counts = {}
    for q in tr:
        counts[q["n"]] = counts.get(q["n"], 0) + 1
    for (n, _), w in zip(si.SERVE_GRIDS, si.SERVE_WEIGHTS):
        assert abs(counts.get(n, 0) / 2000 - w) < 0.04, (n, counts.get(n, 0))
    assert si.serve_trace(si.seed_for(5, 0), 20, rate) == tr[:20]       # a prefix of the same stream
