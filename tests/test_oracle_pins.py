"""Pins of the FP64 oracle's SVT (Eq. 1) and of the Proposition 1 identities.

Each test ties the oracle to something other than itself: a closed form, a
hand-worked fixture in tests/golden/, LAPACK, an invariant of the proximal
operator, or brute force on tiny inputs.
"""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import svt as osvt

RNG = np.random.default_rng(7)


def _svt(a, tau):
    return oracle.svt_definition(np.asarray(a, np.float64), tau)


# ----------------------------------------------------------------- closed forms

@pytest.mark.parametrize("shape", [(5, 5), (7, 4), (4, 7)])
def test_diagonal_closed_form(shape):
    m, n = shape
    k = min(m, n)
    d = RNG.uniform(-2, 2, k)
    a = np.zeros(shape)
    a[np.arange(k), np.arange(k)] = d
    tau = 0.7
    exp = np.zeros(shape)
    exp[np.arange(k), np.arange(k)] = np.sign(d) * np.maximum(np.abs(d) - tau, 0)
    np.testing.assert_allclose(_svt(a, tau), exp, atol=1e-14)


def test_worked_2x2_golden(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "worked_2x2.json")))
    a = np.array(g["A"])
    out, (u, s, v) = oracle.svt_definition(a, g["tau"], return_svd=True)
    np.testing.assert_allclose(s, g["sigma"], rtol=1e-14)
    np.testing.assert_allclose(out, np.array(g["A_tau"]), rtol=1e-13, atol=1e-14)


def _svt_2x2_closed(a, tau):
    """2x2 SVT from the closed-form eigen-decomposition of the symmetric A^T A."""
    p, q, r = a[:, 0] @ a[:, 0], a[:, 0] @ a[:, 1], a[:, 1] @ a[:, 1]
    h = np.hypot(0.5 * (p - r), q)
    lam = [0.5 * (p + r) + h, 0.5 * (p + r) - h]
    out = np.zeros((2, 2))
    for l in lam:
        # eigenvector of [[p,q],[q,r]] for eigenvalue l
        vec = np.array([q, l - p]) if abs(q) > 0 or abs(l - p) > abs(l - r) else np.array([l - r, q])
        if np.linalg.norm(vec) == 0:
            vec = np.array([1.0, 0.0]) if abs(l - p) <= abs(l - r) else np.array([0.0, 1.0])
        vec = vec / np.linalg.norm(vec)
        sig = np.sqrt(max(l, 0.0))
        if sig > tau:
            out += (1 - tau / sig) * np.outer(a @ vec, vec)
    return out


@pytest.mark.parametrize("trial", range(20))
def test_2x2_closed_form(trial):
    rng = np.random.default_rng(100 + trial)
    a = rng.standard_normal((2, 2))
    s = np.linalg.svd(a, compute_uv=False)
    tau = float(rng.uniform(0, 1.2 * s[0]))
    np.testing.assert_allclose(_svt(a, tau), _svt_2x2_closed(a, tau), atol=1e-13)


def test_rank_one():
    u = RNG.standard_normal(9); u /= np.linalg.norm(u)
    v = RNG.standard_normal(6); v /= np.linalg.norm(v)
    for s, tau in [(3.0, 1.0), (0.5, 1.0), (2.0, 0.0)]:
        a = s * np.outer(u, v)
        np.testing.assert_allclose(_svt(a, tau), max(s - tau, 0) * np.outer(u, v), atol=1e-14)


def test_scaled_orthogonal():
    q = np.linalg.qr(RNG.standard_normal((12, 12)))[0]
    for c, tau in [(2.0, 0.5), (0.3, 0.5)]:
        np.testing.assert_allclose(_svt(c * q, tau), max(c - tau, 0) * q, atol=1e-13)


def test_zero_matrix():
    assert np.all(_svt(np.zeros((6, 4)), 0.3) == 0)


# ------------------------------------------------------------------- LAPACK

@pytest.mark.parametrize("shape", [(7, 5), (5, 7), (64, 64), (100, 37), (37, 100), (256, 256),
                                   (512, 512)])
def test_against_lapack(shape):
    rng = np.random.default_rng(sum(shape))
    a = rng.standard_normal(shape)
    u, s, v = np.linalg.svd(a, full_matrices=False)
    tau = float(np.median(s))
    exp = (u * np.maximum(s - tau, 0)[None, :]) @ v
    got = _svt(a, tau)
    assert np.linalg.norm(got - exp) / np.linalg.norm(exp) < 1e-12
    _, s2, _ = oracle.jacobi_svd(a)
    np.testing.assert_allclose(s2, s, rtol=1e-12, atol=1e-13 * s[0])


# ------------------------------------------------------------- invariants

def test_prox_invariants():
    a = RNG.standard_normal((30, 20))
    out, (u, s, v) = oracle.svt_definition(a, 1.5, return_svd=True)
    # ||A - A_tau||_2 = min(tau, sigma_max)
    assert abs(np.linalg.norm(a - out, 2) - min(1.5, s[0])) < 1e-12
    # U1^T (A - A_tau) V1 = tau I on the kept part
    k = int(np.sum(s > 1.5))
    np.testing.assert_allclose(u[:, :k].T @ (a - out) @ v[:, :k], 1.5 * np.eye(k), atol=1e-12)
    # tau above sigma_max gives 0
    assert np.abs(_svt(a, 1.01 * s[0])).max() < 1e-13


def test_homogeneity_orthogonal_transpose():
    a = RNG.standard_normal((15, 11))
    tau = 1.1
    base = _svt(a, tau)
    np.testing.assert_allclose(_svt(2.5 * a, 2.5 * tau), 2.5 * base, atol=1e-12)
    q1 = np.linalg.qr(RNG.standard_normal((15, 15)))[0]
    q2 = np.linalg.qr(RNG.standard_normal((11, 11)))[0]
    np.testing.assert_allclose(_svt(q1 @ a @ q2.T, tau), q1 @ base @ q2.T, atol=1e-12)
    np.testing.assert_allclose(_svt(a.T, tau), base.T, atol=1e-13)


@pytest.mark.parametrize("shape", [(2, 2), (3, 2)])
def test_brute_force_objective(shape):
    """A_tau minimises 1/2||X - A||_F^2 + tau ||X||_* (the nuclear-norm prox)."""
    rng = np.random.default_rng(11)
    for _ in range(5):
        a = rng.standard_normal(shape)
        tau = float(rng.uniform(0.1, 1.0))
        obj = lambda x: 0.5 * np.sum((x - a) ** 2) + tau * np.sum(np.linalg.svd(x, compute_uv=False))
        best = obj(_svt(a, tau))
        pert = rng.standard_normal((10000,) + shape) * rng.uniform(1e-4, 0.5, (10000, 1, 1))
        vals = [obj(_svt(a, tau) + p) for p in pert]
        assert best <= min(vals) + 1e-12


# -------------------------------------------------- Proposition 1 identities

@pytest.mark.parametrize("shape", [(40, 25), (25, 40), (30, 30)])
def test_prop1_identities(shape):
    rng = np.random.default_rng(3)
    a = rng.standard_normal(shape)
    s = np.linalg.svd(a, compute_uv=False)
    tau = float(0.5 * (s[len(s) // 2] + s[len(s) // 2 + 1]))
    exact, (u, sig, v) = oracle.svt_definition(a, tau, return_svd=True)
    p = osvt.polar_from_svd(u, v)
    m, n = shape
    if m >= n:
        s_right = osvt.sign_of_shifted_gram(v, sig, tau * tau)
        assert np.linalg.norm(osvt.prop1(a, p, s_right, tau) - exact) < 1e-12 * np.linalg.norm(exact)
        assert np.linalg.norm(osvt.prop1_factored(a, p, s_right, tau) - exact) < 1e-12 * np.linalg.norm(exact)
    else:
        s_left = osvt.sign_of_shifted_gram(u, sig, tau * tau)
        assert np.linalg.norm(osvt.prop1_footnote(a, p, s_left, tau) - exact) < 1e-12 * np.linalg.norm(exact)
        # the wide case is the tall case of A^T, transposed
        assert np.linalg.norm(osvt.prop1_factored(a.T, p.T, s_left, tau).T - exact) < 1e-12 * np.linalg.norm(exact)


def test_shift_is_tau_squared(golden_dir):
    """Reading: the Gram matrix is shifted by tau^2 (code listing), not tau (proposition as printed)."""
    g = json.load(open(os.path.join(golden_dir, "shift_tau_squared.json")))
    a = np.array(g["A"]); tau = g["tau"]
    np.testing.assert_allclose(_svt(a, tau), np.array(g["A_tau"]), atol=1e-15)
    u, s, v = oracle.jacobi_svd(a)
    p = osvt.polar_from_svd(u, v)
    s2 = osvt.sign_of_shifted_gram(v, s, tau * tau)
    np.testing.assert_allclose(s2, np.array(g["S_tau_squared_shift"]), atol=1e-15)
    np.testing.assert_allclose(osvt.prop1(a, p, s2, tau), np.array(g["A_tau"]), atol=1e-15)
    s1 = osvt.sign_of_shifted_gram(v, s, tau)
    np.testing.assert_allclose(osvt.prop1(a, p, s1, tau), np.array(g["result_with_tau_shift"]), atol=1e-15)


def test_corollary_rank_r():
    """Corollary 1 with descending sigma: tau between sigma_{r+1} and sigma_r gives [A]_r."""
    a = RNG.standard_normal((20, 14))
    u, s, v = oracle.jacobi_svd(a)
    r = 5
    tau = 0.5 * (s[r - 1] + s[r])
    sgn = osvt.sign_of_shifted_gram(v, s, tau * tau)
    np.testing.assert_allclose(osvt.corollary_rank_r(a, sgn), oracle.best_rank_r(a, r), atol=1e-12)
    # Eckart-Young against LAPACK
    uu, ss, vv = np.linalg.svd(a, full_matrices=False)
    np.testing.assert_allclose(oracle.best_rank_r(a, r), (uu[:, :r] * ss[:r]) @ vv[:r], atol=1e-12)


def test_rank_deficient_any_partial_isometry():
    """For rank-deficient A, P is not unique, but (I + S) annihilates the difference."""
    rng = np.random.default_rng(5)
    a = rng.standard_normal((12, 4)) @ rng.standard_normal((4, 9))  # rank 4, 12 x 9
    tau = 0.8
    exact, (u, s, v) = oracle.svt_definition(a, tau, return_svd=True)
    assert s[4] < 1e-12
    p1 = u[:, :4] @ v[:, :4].T  # partial isometry
    q = np.linalg.qr(rng.standard_normal((12, 12)))[0]
    # another valid polar factor: any map of the null space of A into range(A)^perp
    p2 = p1 + (np.eye(12) - u[:, :4] @ u[:, :4].T) @ q[:, :5] @ v[:, 4:].T
    sgn = osvt.sign_of_shifted_gram(v, s, tau * tau)
    for p in (p1, p2):
        np.testing.assert_allclose(osvt.prop1_factored(a, p, sgn, tau), exact, atol=1e-12)


# ------------------------------------------------ gap and the error metric's readings

def test_gap_closed_form_on_diagonal_spectra():
    """gap(tau) = min_i |sigma_i - tau| / sigma_max, with sigma read off the Jacobi SVD of
    a diagonal matrix (so the values are exact). The nearest value sits above tau in the
    first case and below it in the second; sigma_max differs from sigma_min in both, so
    dividing by the wrong extreme, or taking the max distance, changes the value."""
    for diag, tau, want in (([0.1, 1.0, 0.32, 0.5], 0.3, 0.02 / 1.0),
                            ([2.0, 0.28, 0.9, 0.05], 0.3, 0.02 / 2.0),
                            ([4.0, 1.0], 0.0, 1.0 / 4.0),
                            ([3.0, 1.0], 5.0, 2.0 / 3.0)):
        a = np.diag(np.array(diag, np.float64))
        _, s, _ = oracle.jacobi_svd(a)
        assert oracle.gap(s, tau) == pytest.approx(want, rel=1e-12), (diag, tau)
    # tau on a singular value: zero gap
    assert oracle.gap(np.array([1.0, 0.5]), 0.5) == 0.0
    # the zero spectrum has no scale: nothing binds there
    assert oracle.gap(np.zeros(3), 0.2) == float("inf")


def test_gap_gates_the_tier_tolerance_on_the_64x64_recipe():
    """The 64 x 64 recipe puts no singular value in [0.25, 0.35] around tau = 0.3 with
    sigma_max = 1, so its gap is at least 0.05 (Section 3's workloads; the 5 % rule)."""
    import svt_workloads as wl
    _, s, _ = oracle.jacobi_svd(wl.spectrum_64().astype(np.float64))
    g = oracle.gap(s, 0.3)
    assert 0.05 <= g <= 0.07, g


def test_relerr_zero_result_is_relative_to_A():
    """Reading of the error metric when A_tau = 0 (tau >= sigma_max): the error is taken
    relative to ||A||_F. A = diag(3, 4) has ||A||_F = 5; an approximation diag(0.3, 0.4)
    of the zero result is 0.5 / 5 = 0.1 off."""
    a = np.diag([3.0, 4.0])
    exact = _svt(a, 4.5)
    assert np.all(exact == 0.0)
    approx = np.diag([0.3, 0.4])
    assert oracle.relerr(approx, exact, a) == pytest.approx(0.1, rel=1e-15)
    with pytest.raises(ValueError):
        oracle.relerr(approx, exact)
    # both A and the result zero: the absolute norm of the approximation
    assert oracle.relerr(approx, np.zeros((2, 2)), np.zeros((2, 2))) == pytest.approx(0.5)
    # a nonzero result uses its own norm, whatever A is: ||(1, 0) - (1, 1)|| / ||(1, 1)||
    assert oracle.relerr(np.diag([1.0, 0.0]), np.eye(2), a) == pytest.approx(1 / np.sqrt(2))
