"""Nuclear-norm matrix completion by proximal gradient, with SVT by definition.

TEST INFRASTRUCTURE ONLY (see the package docstring). FP64 NumPy on the host.

Section 2 of the paper motivates singular value soft-thresholding (Eq. 1) as
the proximal operator of tau ||.||_* inside proximal gradient methods. The
problem here is

    minimise F(X) = 1/2 ||P_Omega(X - M)||_F^2 + lambda ||X||_*,

P_Omega keeping the observed entries. Its smooth part has gradient
P_Omega(X - M), Lipschitz constant 1, so the proximal-gradient step with step
h in (0, 1] is

    Z = X + h P_Omega(M - X),   X <- A_{h lambda}(Z),

and F does not increase along the iterates. A minimiser X* is characterised by
G = P_Omega(M - X*) lying in lambda times the subdifferential of ||.||_* at X*:
||G||_2 <= lambda and <G, X*> = lambda ||X*||_*.
"""
from __future__ import annotations

import numpy as np

from .native import jacobi_svd
from .svt import svt_definition


def objective(x: np.ndarray, m: np.ndarray, mask: np.ndarray, lam: float) -> float:
    """F(X) = 1/2 ||P_Omega(X - M)||_F^2 + lambda ||X||_* (nuclear norm from the Jacobi SVD)."""
    obs = mask != 0
    r = np.where(obs, x - m, 0.0)
    _, s, _ = jacobi_svd(np.asarray(x, dtype=np.float64))
    return 0.5 * float(np.sum(r * r)) + lam * float(np.sum(s))


def prox_grad_step(x: np.ndarray, m: np.ndarray, mask: np.ndarray, lam: float,
                   step: float = 1.0) -> np.ndarray:
    """One step: Z = X + h P_Omega(M - X), then A_{h lambda}(Z) by Eq. 1."""
    obs = mask != 0
    z = np.where(obs, x + step * (m - x), x)
    return svt_definition(z, step * lam)


def complete(m: np.ndarray, mask: np.ndarray, lam: float, steps: int, step: float = 1.0,
             x0: np.ndarray | None = None, history: bool = False):
    """`steps` proximal-gradient steps from x0 (zeros if None). With history=True also
    returns F after every step."""
    m = np.asarray(m, dtype=np.float64)
    x = np.zeros_like(m) if x0 is None else np.asarray(x0, dtype=np.float64).copy()
    objs = []
    for _ in range(int(steps)):
        x = prox_grad_step(x, m, mask, lam, step)
        if history:
            objs.append(objective(x, m, mask, lam))
    return (x, objs) if history else x


def kkt_residuals(x: np.ndarray, m: np.ndarray, mask: np.ndarray, lam: float):
    """Optimality of X for F: returns (||G||_2 / lambda - 1, |<G, X> - lambda ||X||_*| /
    (lambda ||X||_*)) with G = P_Omega(M - X); both are <= 0 / 0 at a minimiser."""
    obs = mask != 0
    g = np.where(obs, m - x, 0.0)
    _, sg, _ = jacobi_svd(g)
    _, sx, _ = jacobi_svd(np.asarray(x, dtype=np.float64))
    nuc = float(np.sum(sx))
    inner = float(np.sum(g * x))
    return float(sg.max()) / lam - 1.0, abs(inner - lam * nuc) / max(lam * nuc, 1e-300)


def complete_continuation(m: np.ndarray, mask: np.ndarray, lam: float, lam0: float,
                          eta: float, tol: float, max_steps: int, stage_steps: int = 0,
                          step: float = 1.0, x0: np.ndarray | None = None):
    """Proximal gradient with lambda continuation and a stopping test on the iterates.

    Stage k (k = 0, 1, ...) solves at lambda_k = max(lam, lam0 eta^k); the stage whose
    lambda_k equals lam is the last. Each stage runs proximal-gradient steps until the
    relative change rho = ||X_new - X_old||_F / ||P_Omega(M)||_F (measured against the
    data's scale, so that it stays meaningful when the iterate is zero or nearly so; 0
    when both norms are zero, infinity when only the data's is) is <= tol, or until it
    has run stage_steps steps (non-final stages only; 0 = no cap). The run ends when the
    last stage stops or after max_steps steps in total.

    At a fixed lambda the step map is non-expansive, so ||X_new - X_old||_F never grows
    within a stage, and a small change bounds the optimality residual of X_new (see the
    tests). Returns (X, info) with info = {"steps", "stages", "rel_change" (of the last
    step), "lambdas", "changes" (||X_new - X_old||_F), "rhos" (the relative changes) and
    "stage_of_step", each per step}.
    """
    if lam0 < lam:
        raise ValueError("lam0 must be >= lam")
    if lam0 > lam and not (0.0 < eta < 1.0):
        raise ValueError("eta must lie in (0, 1) when lam0 > lam")
    m = np.asarray(m, dtype=np.float64)
    x = np.zeros_like(m) if x0 is None else np.asarray(x0, dtype=np.float64).copy()
    scale = float(np.linalg.norm(np.where(mask != 0, m, 0.0)))
    info = {"steps": 0, "stages": 0, "rel_change": 0.0, "lambdas": [], "changes": [],
            "rhos": [], "stage_of_step": []}
    k = 0
    while info["steps"] < max_steps:
        lam_k = max(lam, lam0 * eta ** k) if lam0 > lam else lam
        last = lam_k == lam
        info["stages"] += 1
        taken = 0
        while info["steps"] < max_steps:
            x_new = prox_grad_step(x, m, mask, lam_k, step)
            d = float(np.linalg.norm(x_new - x))
            rho = d / scale if scale > 0 else (0.0 if d == 0 else np.inf)
            x = x_new
            taken += 1
            info["steps"] += 1
            info["rel_change"] = rho
            info["lambdas"].append(lam_k)
            info["changes"].append(d)
            info["rhos"].append(rho)
            info["stage_of_step"].append(k)
            if rho <= tol or (not last and stage_steps > 0 and taken >= stage_steps):
                break
        if last:
            break
        k += 1
    return x, info
