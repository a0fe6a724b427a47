"""Pins of the oracle's proximal-gradient matrix completion (oracle/completion.py).

Each pin is fixed by the mathematics of the problem, not by the oracle's own
formulas: full observation reduces a step to Eq. 1 on M (closed form for a
diagonal M), lambda = 0 reproduces M, F is non-increasing for steps in (0, 1]
(a sign error in the gradient step makes it increase), the limit satisfies the
optimality conditions ||G||_2 <= lambda, <G, X> = lambda ||X||_* (a wrong lambda
scaling breaks the equality), and brute-force perturbations of the limit never
lower F (convexity: a local minimum is global).
"""
import numpy as np
import pytest

from oracle import completion as oc


def _instance(m, n, rank, frac, seed):
    rng = np.random.default_rng(seed)
    mat = rng.standard_normal((m, rank)) @ rng.standard_normal((rank, n))
    mask = (rng.uniform(size=(m, n)) < frac).astype(np.uint8)
    return mat, mask


def test_full_mask_step_is_soft_threshold_of_m():
    """Omega = everything, h = 1: Z = M, so one step from any X is A_lambda(M); for a
    diagonal M that is sign(d) max(|d| - lambda, 0) on the diagonal."""
    d = np.array([3.0, -1.5, 0.4, -0.05, 2.2])
    m = np.diag(d)
    mask = np.ones_like(m, dtype=np.uint8)
    x0 = np.random.default_rng(1).standard_normal(m.shape)
    lam = 0.5
    x1 = oc.prox_grad_step(x0, m, mask, lam)
    expect = np.diag(np.sign(d) * np.maximum(np.abs(d) - lam, 0.0))
    assert np.max(np.abs(x1 - expect)) < 1e-12


def test_lambda_zero_full_mask_reproduces_m():
    m, _ = _instance(9, 7, 3, 1.0, 2)
    mask = np.ones_like(m, dtype=np.uint8)
    x1 = oc.prox_grad_step(np.zeros_like(m), m, mask, 0.0)
    assert np.max(np.abs(x1 - m)) < 1e-12 * np.abs(m).max()


def test_unobserved_entries_do_not_enter_the_step():
    """Changing M off Omega changes nothing."""
    m, mask = _instance(10, 8, 2, 0.5, 3)
    m2 = m.copy()
    m2[mask == 0] += 100.0
    x0 = np.random.default_rng(4).standard_normal(m.shape)
    a = oc.prox_grad_step(x0, m, mask, 0.3)
    b = oc.prox_grad_step(x0, m2, mask, 0.3)
    assert np.max(np.abs(a - b)) < 1e-12


@pytest.mark.parametrize("step", [1.0, 0.5])
def test_objective_non_increasing(step):
    m, mask = _instance(20, 16, 2, 0.4, 5)
    lam = 0.1 * np.linalg.norm(m * mask, 2)
    _, objs = oc.complete(m, mask, lam, 40, step=step, history=True)
    f0 = oc.objective(np.zeros_like(m), m, mask, lam)
    seq = [f0] + objs
    for a, b in zip(seq, seq[1:]):
        assert b <= a * (1 + 1e-12) + 1e-12
    assert seq[-1] < seq[0]


def test_limit_satisfies_optimality_conditions():
    m, mask = _instance(12, 10, 2, 0.6, 6)
    lam = 0.2 * np.linalg.norm(m * mask, 2)
    x = oc.complete(m, mask, lam, 3000)
    gnorm, gap = oc.kkt_residuals(x, m, mask, lam)
    assert gnorm < 1e-6, gnorm
    assert gap < 1e-6, gap


def test_limit_is_a_minimum_under_random_perturbations():
    m, mask = _instance(5, 4, 1, 0.6, 7)
    lam = 0.15 * np.linalg.norm(m * mask, 2)
    x = oc.complete(m, mask, lam, 4000)
    f = oc.objective(x, m, mask, lam)
    rng = np.random.default_rng(8)
    for scale in (1e-1, 1e-2, 1e-3):
        for _ in range(300):
            assert oc.objective(x + scale * rng.standard_normal(x.shape), m, mask, lam) >= f - 1e-10
