"""Pins of the oracle's odd-polynomial schedules (Remez) and its spectral model."""
import math

import numpy as np
import pytest

import oracle
from oracle import schedule as sch
from oracle import spectral

import svt_workloads as wl


def _cubic_closed_form(ell):
    """Minimax odd cubic a x + b x^3 for 1 on [ell, 1], derived by hand.

    Equioscillation at ell, x*, 1 with p'(x*) = 0: from p(ell) = p(1),
    a = -b (1 + ell + ell^2), x*^2 = (1 + ell + ell^2)/3, and p(ell) + p(x*) = 2 gives
    b = -2 / ((2/3)(1 + ell + ell^2) x* + ell + ell^2)."""
    q = 1 + ell + ell * ell
    xs = math.sqrt(q / 3)
    b = -2.0 / ((2.0 / 3.0) * q * xs + ell + ell * ell)
    a = -b * q
    err = 1 - (a + b)
    return (a, b), err


@pytest.mark.parametrize("ell", [1e-3, 0.05, 0.3, 0.9])
def test_remez_cubic_closed_form(ell):
    (a, b), err = _cubic_closed_form(ell)
    coef, e = sch.remez_odd(ell, 1.0, 2)
    np.testing.assert_allclose(coef, (a, b), rtol=1e-10)
    assert abs(e - err) < 1e-10


@pytest.mark.parametrize("lo,hi", [(1e-3, 1.0), (0.2, 1.3), (0.9, 1.1)])
def test_remez_equioscillates(lo, hi):
    coef, e = sch.remez_odd(lo, hi, 3)
    grid = np.linspace(lo, hi, 400001)
    err = 1 - sch.eval_odd(coef, grid)
    assert abs(np.max(np.abs(err)) - e) < 1e-9 * max(e, 1e-3)
    # four alternation points: ends and two interior extrema, signs + - + -
    crit = sch._critical_points(coef, lo, hi)
    pts = np.array([lo] + crit + [hi])
    assert len(pts) == 4
    vals = 1 - sch.eval_odd(coef, pts)
    np.testing.assert_allclose(np.abs(vals), e, rtol=1e-9)
    assert np.all(np.sign(vals) == np.array([1, -1, 1, -1]))


def test_remez_scaling_covariance():
    """The minimax poly on [l, u] is the one on [l/u, 1] evaluated at x/u:
    coefficients scale as (a/u, b/u^3, c/u^5)."""
    (c1, e1) = sch.remez_odd(0.01, 1.0, 3)
    (c2, e2) = sch.remez_odd(0.01 * 2.5, 2.5, 3)
    np.testing.assert_allclose(c2, (c1[0] / 2.5, c1[1] / 2.5 ** 3, c1[2] / 2.5 ** 5), rtol=1e-9)
    assert abs(e1 - e2) < 1e-12


def test_narrow_interval_limit_is_ns_quintic():
    """As [1-h, 1+h] shrinks, the minimax quintic tends to (15/8, -5/4, 3/8)."""
    prev = None
    for h in (0.2, 0.05, 0.01):
        coef, _ = sch.remez_odd(1 - h, 1 + h, 3)
        d = np.max(np.abs(np.array(coef) - np.array(sch.NS5)))
        if prev is not None:
            assert d < prev
        prev = d
    assert prev < 1e-3


@pytest.mark.parametrize("delta", [0.0, 0.01])
def test_pe5_composition_on_grid(delta):
    """Composition of the schedule maps [l0, 1] into the interval the schedule predicts."""
    coefs, bounds = sch.pe5_schedule(12, 1e-3, delta)
    x = np.concatenate([np.geomspace(1e-3, 1, 20001), np.linspace(1e-3, 1 + delta, 20001)])
    y = x.copy()
    for t, c in enumerate(coefs):
        y = sch.eval_odd(c, y)
        if t + 1 < len(bounds):
            lo, hi = bounds[t + 1]
            assert y.min() >= lo - 1e-9 and y.max() <= hi * (1 + delta) + 1e-9
    assert np.max(np.abs(y - 1)) < 1e-6
    # odd: negative inputs map to the negative of the positive ones
    np.testing.assert_allclose(sch.compose(coefs, -x[:100]), -sch.compose(coefs, x[:100]), rtol=1e-15)


def test_ns3_is_newton_schulz():
    assert sch.ns3_schedule(3) == [(1.5, -0.5)] * 3
    # x -> 3/2 x - 1/2 x^3 fixes 1 with zero derivative (quadratic convergence)
    x = 1 + 1e-4
    assert abs(sch.eval_odd((1.5, -0.5), x) - 1) < 2e-8


# ------------------------------------------------------------ spectral model

@pytest.mark.parametrize("shape", [(24, 16), (16, 24), (20, 20)])
@pytest.mark.parametrize("norm", ["fro", "gram"])
@pytest.mark.parametrize("polish", [True, False])
def test_spectral_model_matches_plain_iteration(shape, norm, polish):
    """Unconverged (3 steps): the scalar model must equal the FP64 matrix iteration."""
    rng = np.random.default_rng(21)
    a = rng.standard_normal(shape)
    u, s, v = oracle.jacobi_svd(a)
    tau = float(s[len(s) // 3])
    cp, _ = sch.pe5_schedule(3, 1e-2, 0.01)
    cs = sch.ns3_schedule(4)
    pred = spectral.predict(u, s, v, tau, cp, cs, norm, norm, polish)
    plain = oracle.svt_polar_plain(a, tau, cp, cs, norm, norm, polish)
    assert np.linalg.norm(pred - plain) <= 1e-12 * np.linalg.norm(plain)


def test_converged_model_is_the_definition():
    a = wl.spectrum_64().astype(np.float64)
    exact, (u, s, v) = oracle.svt_definition(a, 0.3, return_svd=True)
    cp, _ = sch.pe5_schedule(20, 1e-3, 0.0)
    pred = spectral.predict(u, s, v, 0.3, cp, cp, "gram", "gram")
    assert oracle.relerr(pred, exact) < 1e-14
    ns = sch.ns3_schedule(30)
    assert oracle.relerr(oracle.svt_polar_plain(a, 0.3, ns, ns, "fro", "fro"), exact) < 1e-12
