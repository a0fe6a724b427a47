"""SVT by definition, the Proposition 1 identities, and the plain polar iteration.

TEST INFRASTRUCTURE ONLY (see the package docstring). Everything here is FP64
NumPy on the host; matrix products are NumPy matmuls, the SVD is the Jacobi
routine of ``native.py``.

Citations are to the paper (Becker, "Singular value soft-thresholding via the
polar decomposition"): Eq. 1 (the SVT definition), Proposition 1 and its
footnote (the polar forms), the proof of Proposition 1 (the spectral forms of P
and S), Corollary 1 (best rank-r approximation) and Section 4 (the code listing,
which shifts the Gram matrix by tau**2 and branches on the shape).
"""
from __future__ import annotations

import numpy as np

from .native import jacobi_svd


def svt_definition(a: np.ndarray, tau: float, return_svd: bool = False):
    """Eq. 1: A_tau = U max(Sigma - tau I, 0) V^T, accumulated in FP64.

    U, sigma, V come from the FP64 one-sided Jacobi SVD; the thresholded values
    multiply U's columns and the product with V^T is a NumPy matmul.
    """
    if tau < 0 or not np.isfinite(tau):
        raise ValueError("tau must be finite and >= 0")
    u, s, v = jacobi_svd(a)
    shrunk = np.maximum(s - tau, 0.0)
    out = (u * shrunk[None, :]) @ v.T
    if return_svd:
        return out, (u, s, v)
    return out


def best_rank_r(a: np.ndarray, r: int) -> np.ndarray:
    """Truncated SVD sum_{i<=r} sigma_i u_i v_i^T (Eckart-Young), from the Jacobi SVD."""
    u, s, v = jacobi_svd(a)
    return (u[:, :r] * s[None, :r]) @ v[:, :r].T


def polar_from_svd(u: np.ndarray, v: np.ndarray) -> np.ndarray:
    """P = U V^T (Section 2: the polar factor from the SVD)."""
    return u @ v.T


def sign_of_shifted_gram(v: np.ndarray, s: np.ndarray, shift: float) -> np.ndarray:
    """S = polar(A^T A - shift I) = V sign(sigma^2 - shift) V^T for square V.

    This is the spectral form used in the proof of Proposition 1
    (S = V1 V1^T - V2 V2^T). An eigenvalue exactly 0 maps to 0."""
    return (v * np.sign(s * s - shift)[None, :]) @ v.T


def prop1(a, p, s, tau):
    """Proposition 1: A_tau = 1/2 (A + A S) - tau/2 (P + P S), S = polar(A^T A - tau^2 I)."""
    return 0.5 * (a + a @ s) - 0.5 * tau * (p + p @ s)


def prop1_footnote(a, p, s_left, tau):
    """Footnote of Proposition 1: A_tau = 1/2 (A + S A) - tau/2 (P + S P),
    S = polar(A A^T - tau^2 I)."""
    return 0.5 * (a + s_left @ a) - 0.5 * tau * (p + s_left @ p)


def prop1_factored(a, p, s, tau):
    """The factored form 1/2 (A - tau P)(I + S), algebraically equal to Proposition 1."""
    n = s.shape[0]
    return 0.5 * (a - tau * p) @ (np.eye(n) + s)


def corollary_rank_r(a, s):
    """Corollary 1: [A]_r = 1/2 (A + A S) with S the sign of A^T A - tau^2 I, tau in
    the gap between sigma_{r+1} and sigma_r."""
    return 0.5 * (a + a @ s)


def relerr(approx: np.ndarray, exact: np.ndarray, a: np.ndarray | None = None) -> float:
    """Relative Frobenius error ||approx - exact||_F / ||exact||_F (Fig. 1 caption).

    When the exact result is zero (tau >= sigma_max) the error is taken relative
    to ||A||_F instead, which needs ``a``."""
    approx = np.asarray(approx, np.float64)
    exact = np.asarray(exact, np.float64)
    den = np.linalg.norm(exact)
    if den == 0.0:
        if a is None:
            raise ValueError("exact result is zero: pass A for the absolute reading")
        den = np.linalg.norm(np.asarray(a, np.float64))
        if den == 0.0:
            return float(np.linalg.norm(approx))
    return float(np.linalg.norm(approx - exact) / den)


def gap(sigma: np.ndarray, tau: float) -> float:
    """min_i |sigma_i - tau| / sigma_max: how far tau sits from the spectrum."""
    smax = float(np.max(sigma)) if len(sigma) else 0.0
    if smax == 0.0:
        return float("inf")
    return float(np.min(np.abs(np.asarray(sigma) - tau)) / smax)


# ---------------------------------------------------------------------------
# The method itself, step by step, in plain FP64 matrix arithmetic.
# ---------------------------------------------------------------------------

def _odd_poly_step(x: np.ndarray, coef, gram: np.ndarray | None = None) -> np.ndarray:
    """One odd-polynomial polar step X <- X (c0 I + c1 X^T X + c2 (X^T X)^2 + ...).

    ``coef`` are the coefficients of p(x) = c0 x + c1 x^3 + c2 x^5 + ...; ``gram``
    may pass a precomputed X^T X."""
    y = x.T @ x if gram is None else gram
    n = y.shape[0]
    z = np.zeros((n, n))
    ypow = np.eye(n)
    for c in coef:
        z = z + c * ypow
        ypow = ypow @ y
    return x @ z


def polar_iteration(x0: np.ndarray, schedule, norm: str) -> np.ndarray:
    """Plain polar iteration: normalise X0, then apply each step's odd polynomial.

    norm = "fro":  X <- X0 / ||X0||_F           (||X0||_2 <= ||X0||_F)
    norm = "gram": X <- X0 / ||X0^T X0||_F^{1/2} (||X0||_2^2 = ||X0^T X0||_2 <= ||X0^T X0||_F)
    ``schedule`` is a sequence of coefficient tuples, one per step."""
    x = np.asarray(x0, np.float64)
    if norm == "fro":
        theta = np.linalg.norm(x)
    elif norm == "gram":
        theta = np.sqrt(np.linalg.norm(x.T @ x))
    else:
        raise ValueError(norm)
    if theta == 0.0:
        return np.zeros_like(x)
    x = x / theta
    for coef in schedule:
        x = _odd_poly_step(x, coef)
    return x


def svt_polar_plain(a: np.ndarray, tau: float, sched_p, sched_s, norm_p: str, norm_s: str,
                    polish: bool = True) -> np.ndarray:
    """The method as a plain FP64 matrix computation (Proposition 1, footnote, Section 4).

    1. Branch on shape: A^T A when m >= n, A A^T when n > m (footnote). The wide
       case is the tall case of A^T, transposed back.
    2. P = polar(A) by the odd-polynomial iteration ``sched_p``.
    3. S = polar(A^T A - tau^2 I) by the iteration ``sched_s`` (shift tau^2, as in the
       code listing of Section 4; the proposition as printed writes tau I).
    4. Optional polish: one cubic Newton-Schulz step X(3/2 I - 1/2 X^T X) on each.
    5. A_tau = 1/2 (A - tau P)(I + S).
    """
    a = np.asarray(a, np.float64)
    m, n = a.shape
    if n > m:
        return svt_polar_plain(a.T, tau, sched_p, sched_s, norm_p, norm_s, polish).T
    p = polar_iteration(a, sched_p, norm_p)
    g = a.T @ a - (tau * tau) * np.eye(n)
    s = polar_iteration(g, sched_s, norm_s)
    if polish:
        p = _odd_poly_step(p, (1.5, -0.5))
        s = _odd_poly_step(s, (1.5, -0.5))
    return prop1_factored(a, p, s, tau)
