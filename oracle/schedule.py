"""Odd-polynomial polar schedules, derived independently for the oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper runs its polar decompositions with Polar Express (Section 3, which
cites Amsel et al. 2025) and Newton-Schulz (Section 1). The third-party
coefficient table is not part of the paper, so the schedule is derived here
from the published method itself:

* Polar Express (``pe5``): step t applies the odd quintic p_t(x) = a x + b x^3 + c x^5
  that minimises max |1 - p_t(x)| over [l_t, (1 + delta) u_t]; the next interval
  is the image [1 - E_t, 1 + E_t], where E_t is that minimax error. The first
  interval is [l_0, 1]. The widening by (1 + delta) leaves headroom for rounding.
  Once the design interval is narrower than ``SWITCH_WIDTH`` the minimax problem
  is ill-conditioned in FP64; from then on the step is the Newton-Schulz quintic
  (15/8, -5/4, 3/8), the limit of the minimax quintic as the interval shrinks to
  the point 1 (p(1) = 1, p'(1) = p''(1) = 0).
* Newton-Schulz (``ns3``): the cubic (3/2, -1/2) at every step.

The minimax polynomial is found by the Remez exchange algorithm: solve for the
coefficients and the levelled error on a reference of d + 1 points, move the
reference to the extrema of the error (the interval's ends and the roots of
p'(x), a polynomial in x^2), and repeat until the error levels.
"""
from __future__ import annotations

import numpy as np

SWITCH_WIDTH = 1e-3
NS5 = (15.0 / 8.0, -10.0 / 8.0, 3.0 / 8.0)
NS3 = (1.5, -0.5)


def _eval_odd(coef, x):
    x = np.asarray(x, np.float64)
    x2 = x * x
    out = np.zeros_like(x)
    xp = x.copy()
    for c in coef:
        out = out + c * xp
        xp = xp * x2
    return out


def eval_odd(coef, x):
    """p(x) = sum_j coef[j] x^(2j+1)."""
    return _eval_odd(coef, x)


def _critical_points(coef, lo, hi):
    """Roots of p'(x) = sum_j (2j+1) coef[j] x^(2j) inside (lo, hi)."""
    # p'(x) as a polynomial in y = x^2, highest power first for numpy.roots.
    dcoef = [(2 * j + 1) * c for j, c in enumerate(coef)][::-1]
    while len(dcoef) > 1 and dcoef[0] == 0.0:
        dcoef = dcoef[1:]
    if len(dcoef) <= 1:
        return []
    ys = np.roots(dcoef)
    out = []
    for y in ys:
        if abs(y.imag) > 1e-12 * max(1.0, abs(y.real)) or y.real <= 0:
            continue
        x = float(np.sqrt(y.real))
        if lo < x < hi:
            out.append(x)
    return sorted(out)


def remez_odd(lo: float, hi: float, ncoef: int = 3, iters: int = 200, tol: float = 1e-15):
    """Minimax odd polynomial of degree 2*ncoef - 1 approximating 1 on [lo, hi].

    Returns (coefficients, E) with E = max_{[lo,hi]} |1 - p(x)|.
    """
    if not (0.0 < lo < hi):
        raise ValueError("need 0 < lo < hi")
    npts = ncoef + 1
    # Initial reference: Chebyshev extrema mapped to [lo, hi].
    k = np.arange(npts)
    ref = 0.5 * (lo + hi) - 0.5 * (hi - lo) * np.cos(np.pi * k / (npts - 1))
    coef = None
    lev = 0.0
    for _ in range(iters):
        mat = np.zeros((npts, npts))
        for i, x in enumerate(ref):
            for j in range(ncoef):
                mat[i, j] = x ** (2 * j + 1)
            mat[i, ncoef] = (-1.0) ** i
        sol = np.linalg.solve(mat, np.ones(npts))
        coef = sol[:ncoef]
        lev = abs(sol[ncoef])
        cand = [lo] + _critical_points(coef, lo, hi) + [hi]
        if len(cand) != npts:
            # Fall back to a dense search for the alternating extrema.
            grid = np.linspace(lo, hi, 200001)
            err = 1.0 - _eval_odd(coef, grid)
            idx = [0]
            for i in range(1, len(grid) - 1):
                if (err[i] - err[i - 1]) * (err[i + 1] - err[i]) <= 0:
                    idx.append(i)
            idx.append(len(grid) - 1)
            cand = [float(grid[i]) for i in idx]
            if len(cand) > npts:
                # Keep the npts largest |err| points in order (simple, adequate here).
                order = sorted(sorted(range(len(cand)), key=lambda i: -abs(err[idx[i]]))[:npts])
                cand = [cand[i] for i in order]
            elif len(cand) < npts:
                break
        new_ref = np.array(cand)
        errs = 1.0 - _eval_odd(coef, new_ref)
        emax = float(np.max(np.abs(errs)))
        if np.allclose(new_ref, ref, rtol=0, atol=tol * hi) or emax - lev <= tol * max(lev, 1e-300):
            ref = new_ref
            break
        ref = new_ref
    # Report the true maximum error on the final coefficients.
    cand = [lo] + _critical_points(coef, lo, hi) + [hi]
    emax = float(np.max(np.abs(1.0 - _eval_odd(coef, np.array(cand)))))
    return tuple(float(c) for c in coef), max(emax, lev)


def pe5_schedule(steps: int, ell0: float = 1e-3, delta: float = 0.0):
    """Polar-Express-style quintic schedule: list of (a, b, c) and the interval
    bounds [(l_t, u_t)] each step was designed for (before widening)."""
    lo, hi = float(ell0), 1.0
    coefs, bounds = [], []
    for _ in range(steps):
        dhi = hi * (1.0 + delta)
        bounds.append((lo, hi))
        if dhi - lo < SWITCH_WIDTH:
            coef = NS5
            xs = np.array([lo] + _critical_points(coef, lo, dhi) + [dhi])
            ys = _eval_odd(coef, xs)
            lo, hi = float(np.min(ys)), float(np.max(ys))
        else:
            coef, err = remez_odd(lo, dhi, 3)
            lo, hi = 1.0 - err, 1.0 + err
        coefs.append(tuple(coef))
    return coefs, bounds


def ns3_schedule(steps: int):
    """Newton-Schulz cubic schedule: (3/2, -1/2) at every step."""
    return [NS3] * steps


def compose(coefs, x):
    """Apply the schedule's polynomials in order to scalars x."""
    y = np.asarray(x, np.float64)
    for c in coefs:
        y = _eval_odd(c, y)
    return y
