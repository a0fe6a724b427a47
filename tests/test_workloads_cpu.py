"""Host checks of the seeded input recipes that have a closed form to meet: the
Marchenko-Pastur quantiles behind the known-SVD stand-ins of the benchmark matrices."""
import math

import numpy as np

import svt_workloads as wl


def test_mp_quantiles_square_case_is_the_quarter_circle():
    """For n x n N(0, 1/n) entries the Marchenko-Pastur singular-value law is the
    quarter circle on [0, 2], whose distribution function has a closed form."""
    for n in (64, 1000):
        q = wl.quarter_circle_sigma(n)
        m = wl.mp_noise_sigma(n, n, 1.0 / math.sqrt(n), n)
        assert np.abs(q - m).max() < 1e-6


def test_mp_quantiles_rectangular_edges_and_sampling():
    """Quantiles lie inside the bulk s (sqrt(N) -/+ sqrt(k)) and, largest first, match the
    sorted singular values of a sampled Gaussian matrix of the same shape and scale to a
    few per cent of the edge (finite-size fluctuations)."""
    m, n, s = 1600, 400, 0.01
    q = wl.mp_noise_sigma(m, n, s, n)
    lo, hi = s * (math.sqrt(m) - math.sqrt(n)), s * (math.sqrt(m) + math.sqrt(n))
    assert np.all(np.diff(q) <= 0) and lo < q[-1] and q[0] < hi
    rng = np.random.default_rng(5)
    emp = np.linalg.svd(s * rng.standard_normal((m, n)), compute_uv=False)
    assert np.abs(emp - q).max() < 0.03 * hi
    assert abs(np.median(emp) - np.median(q)) < 0.005 * hi
    # the same law for the wide shape
    assert np.allclose(wl.mp_noise_sigma(n, m, s, n), q)


def test_low_rank_plus_noise_spectrum():
    sig = wl.low_rank_plus_noise_spectrum(8192, 2048, 64, wl.SEED_LOWRANK)
    assert sig.shape == (2048,) and np.all(np.diff(sig) <= 0)
    edge = wl.noise_edge(8192, 2048)
    assert np.sum(sig > edge) <= 64 and np.all(sig[:64] >= 1.0) and sig[0] <= 10.0
    noise = np.sort(sig)[: 2048 - 64]
    assert noise.min() > 0.01 * (math.sqrt(8192) - math.sqrt(2048)) and noise.max() < edge
