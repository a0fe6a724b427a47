"""Exact-arithmetic prediction of the polar-SVT method from the singular values.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Every step of the method is an odd polynomial of the iterate, so it acts on the
singular values alone (proof of Proposition 1: P = U V^T, S = V1 V1^T - V2 V2^T
are spectral functions of A). With A = U diag(sigma) V^T:

* P chain: x0 = sigma / theta_P, then f = p_T(...p_1(x0)) (and the polish step),
  so that P_approx = U diag(f) V^T.
* S chain: the Gram matrix shifted by tau^2 has eigenvalues lam = sigma^2 - tau^2;
  y0 = lam / theta_S, g = composition applied to y0, S_approx = V diag(g) V^T.
* Combine: 1/2 (A - tau P)(I + S) = U diag(1/2 (sigma - tau f)(1 + g)) V^T.

theta is the normalisation: "fro" divides by the Frobenius norm of the chain's
starting matrix, "gram" by ||X0^T X0||_F^{1/2}; both are upper bounds on the
spectral norm, expressed here through sigma.
"""
from __future__ import annotations

import numpy as np

from .schedule import compose, NS3


def _theta(vals: np.ndarray, norm: str) -> float:
    vals = np.asarray(vals, np.float64)
    if norm == "fro":
        return float(np.sqrt(np.sum(vals ** 2)))
    if norm == "gram":
        return float(np.sum(vals ** 4) ** 0.25)
    raise ValueError(norm)


def chain_factors(sigma, tau, sched_p, sched_s, norm_p, norm_s, polish=True):
    """Per singular value: (f_i, g_i) after the P and S chains (and polish)."""
    sigma = np.asarray(sigma, np.float64)
    tp = _theta(sigma, norm_p)
    x0 = sigma / tp if tp > 0 else np.zeros_like(sigma)
    lam = sigma * sigma - tau * tau
    ts = _theta(lam, norm_s)
    y0 = lam / ts if ts > 0 else np.zeros_like(lam)
    f = compose(sched_p, x0)
    g = compose(sched_s, y0)
    if polish:
        f = compose([NS3], f)
        g = compose([NS3], g)
    return f, g


def predicted_values(sigma, tau, sched_p, sched_s, norm_p, norm_s, polish=True):
    """1/2 (sigma - tau f)(1 + g): the singular-value map the method applies."""
    f, g = chain_factors(sigma, tau, sched_p, sched_s, norm_p, norm_s, polish)
    return 0.5 * (np.asarray(sigma, np.float64) - tau * f) * (1.0 + g)


def predict(u, sigma, v, tau, sched_p, sched_s, norm_p, norm_s, polish=True):
    """Predicted output U diag(1/2 (sigma - tau f)(1 + g)) V^T of the method."""
    w = predicted_values(sigma, tau, sched_p, sched_s, norm_p, norm_s, polish)
    return (u * w[None, :]) @ v.T
