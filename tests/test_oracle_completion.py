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


# --- lambda continuation with a stopping test (complete_continuation)
#
# Pins from the mathematics of proximal gradient at a fixed lambda:
# * the step map T is non-expansive (a gradient step of a 1-smooth convex function with
#   h in (0, 1], then a proximal operator), so ||X_{t+1} - X_t|| = ||T X_t - T X_{t-1}||
#   never exceeds ||X_t - X_{t-1}||: the changes do not grow within a stage;
# * with D = X_t - X_{t+1} and r = ||D||_F, prox optimality puts (Z_t - X_{t+1}) / h in
#   lambda d||X_{t+1}||_*, and G = P_Omega(M - X_{t+1}) differs from it by
#   P_Omega(D) - D / h, so ||G||_2 <= lambda + (1 + 1/h) r and
#   |<G, X_{t+1}> - lambda ||X_{t+1}||_*| <= (1 + 1/h) r ||X_{t+1}||_*. A last stage at the
#   wrong lambda, or a wrong sign in the gradient step, breaks these bounds.

def _cont_instance(seed=11):
    m, mask = _instance(14, 11, 2, 0.6, seed)
    s0 = np.linalg.norm(m * mask, 2)
    return m, mask, 0.04 * s0, 0.8 * s0


def test_continuation_changes_do_not_grow_within_a_stage():
    m, mask, lam, lam0 = _cont_instance()
    for step in (1.0, 0.5):
        _, info = oc.complete_continuation(m, mask, lam, lam0, 0.5, 1e-9, 3000, step=step)
        ch, st = info["changes"], info["stage_of_step"]
        for i in range(1, len(ch)):
            if st[i] == st[i - 1]:
                assert ch[i] <= ch[i - 1] * (1 + 1e-9) + 1e-13, (i, ch[i], ch[i - 1])


@pytest.mark.parametrize("step", [1.0, 0.5])
def test_continuation_residual_bounds_at_the_stop(step):
    m, mask, lam, lam0 = _cont_instance(12)
    x, info = oc.complete_continuation(m, mask, lam, lam0, 0.5, 1e-7, 5000, step=step)
    assert info["lambdas"][-1] == lam
    r = info["changes"][-1]
    g = np.where(mask != 0, m - x, 0.0)
    sg = np.linalg.svd(g, compute_uv=False)
    sx = np.linalg.svd(x, compute_uv=False)
    slack = (1 + 1 / step) * r
    assert sg[0] <= lam + slack + 1e-12, (sg[0], lam, slack)
    assert abs(np.sum(g * x) - lam * sx.sum()) <= slack * sx.sum() + 1e-12
    # the bound is not vacuous: the residual is close to lambda at the minimiser
    assert sg[0] >= lam - slack - 1e-9


@pytest.mark.parametrize("tol", [1e-5, 0.05])
def test_continuation_stops_at_the_first_crossing(tol):
    """Every stage ends at the first step whose relative change is <= tol; with the
    loose tolerance some stages end after their first step."""
    m, mask, lam, lam0 = _cont_instance(13)
    _, info = oc.complete_continuation(m, mask, lam, lam0, 0.5, tol, 4000)
    rho, st = np.array(info["rhos"]), np.array(info["stage_of_step"])
    lengths = []
    for k in np.unique(st):
        r = rho[st == k]
        assert r[-1] <= tol
        assert np.all(r[:-1] > tol)
        lengths.append(len(r))
    if tol > 0.01:
        assert min(lengths) == 1, lengths


def test_continuation_stage_lambdas_and_caps():
    m, mask, lam, lam0 = _cont_instance(14)
    eta, cap = 0.5, 3
    _, info = oc.complete_continuation(m, mask, lam, lam0, eta, 0.0, 40, stage_steps=cap)
    lams, st = np.array(info["lambdas"]), np.array(info["stage_of_step"])
    stages = int(np.ceil(np.log(lam / lam0) / np.log(eta))) + 1
    assert info["stages"] == stages
    for k in range(stages):
        assert np.all(lams[st == k] == max(lam, lam0 * eta ** k))
        if k < stages - 1:
            assert np.sum(st == k) == cap
    assert info["steps"] == 40 and np.sum(st == stages - 1) == 40 - cap * (stages - 1)


def test_continuation_reaches_the_cold_start_minimum():
    m, mask, lam, lam0 = _cont_instance(15)
    xc, info = oc.complete_continuation(m, mask, lam, lam0, 0.5, 1e-10, 6000)
    xs = oc.complete(m, mask, lam, 6000)
    fc, fs = oc.objective(xc, m, mask, lam), oc.objective(xs, m, mask, lam)
    assert abs(fc - fs) <= 1e-8 * fs, (fc, fs)


def test_continuation_degenerate_cases():
    m, mask, lam, lam0 = _cont_instance(16)
    x0 = np.random.default_rng(0).standard_normal(m.shape)
    x, info = oc.complete_continuation(m, mask, lam, lam0, 0.5, 1e-6, 0, x0=x0)
    assert info["steps"] == 0 and info["stages"] == 0 and np.array_equal(x, x0)
    # lam0 == lam: a single stage, the plain loop
    x1, info1 = oc.complete_continuation(m, mask, lam, lam, 1.0, 0.0, 7)
    assert info1["stages"] == 1 and info1["steps"] == 7
    assert np.max(np.abs(x1 - oc.complete(m, mask, lam, 7))) == 0.0
    with pytest.raises(ValueError):
        oc.complete_continuation(m, mask, lam, 0.5 * lam, 0.5, 0.0, 3)
    with pytest.raises(ValueError):
        oc.complete_continuation(m, mask, lam, lam0, 1.0, 0.0, 3)


def test_continuation_stops_exactly_when_the_iterate_stays_zero():
    """A stage whose lambda exceeds sigma_max of P_Omega(M) (the first step from X = 0
    thresholds everything) ends after one step with change 0: the zero iterate is that
    stage's fixed point, whatever tol is."""
    m, mask, lam, _ = _cont_instance(17)
    s0 = np.linalg.norm(m * mask, 2)
    x, info = oc.complete_continuation(m, mask, lam, 2.0 * s0, 0.5, 0.0, 50, stage_steps=10)
    st = np.array(info["stage_of_step"])
    assert np.sum(st == 0) == 1 and info["changes"][0] == 0.0 and info["rhos"][0] == 0.0
    # the next stages move
    assert info["changes"][-1] > 0.0 or info["steps"] > 1
