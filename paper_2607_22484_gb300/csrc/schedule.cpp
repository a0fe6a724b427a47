// Polynomial schedules for the polar iterations (host code).
//
// The paper computes both polar factors with Polar Express (Section 3) or
// Newton-Schulz (Section 1): each step applies an odd polynomial to the
// iterate's singular values. The Polar Express coefficient table itself is
// third-party code outside the paper, so the library derives its schedule from
// the method's definition:
//
//   step t uses the odd quintic p(x) = a x + b x^3 + c x^5 minimising
//   max |1 - p(x)| on [l_t, (1 + delta) u_t] (Chebyshev/minimax, solved by the
//   Remez exchange); the next interval is [1 - E_t, 1 + E_t], E_t the levelled
//   error; [l_0, u_0] = [ell0, 1]. Once the design interval is narrower than
//   1e-3 the minimax problem is ill-conditioned in double precision and the
//   step becomes its narrow-interval limit, the Newton-Schulz quintic
//   (15/8, -5/4, 3/8) (p(1) = 1, p'(1) = p''(1) = 0).
//
// Newton-Schulz (NS3) is the cubic (3/2, -1/2, 0) at every step.
#include <algorithm>
#include <cmath>
#include <vector>

#include "svt_internal.h"

namespace svt {

namespace {

constexpr double kSwitchWidth = 1e-3;

double peval(const double c[3], double x)
{
    double x2 = x * x;
    return x * (c[0] + x2 * (c[1] + x2 * c[2]));
}

// Solve the 4 x 4 system m y = rhs by Gaussian elimination with partial pivoting.
bool solve4(double m[4][5], double y[4])
{
    for (int col = 0; col < 4; ++col) {
        int piv = col;
        for (int r = col + 1; r < 4; ++r)
            if (std::fabs(m[r][col]) > std::fabs(m[piv][col]))
                piv = r;
        if (m[piv][col] == 0.0)
            return false;
        if (piv != col)
            for (int k = 0; k < 5; ++k)
                std::swap(m[piv][k], m[col][k]);
        for (int r = col + 1; r < 4; ++r) {
            double f = m[r][col] / m[col][col];
            for (int k = col; k < 5; ++k)
                m[r][k] -= f * m[col][k];
        }
    }
    for (int r = 3; r >= 0; --r) {
        double s = m[r][4];
        for (int k = r + 1; k < 4; ++k)
            s -= m[r][k] * y[k];
        y[r] = s / m[r][r];
    }
    return true;
}

// Interior stationary points of p in (lo, hi): p'(x) = a + 3 b x^2 + 5 c x^4 = 0,
// a quadratic in y = x^2.
std::vector<double> stationary(const double c[3], double lo, double hi)
{
    std::vector<double> ys;
    const double qa = 5.0 * c[2], qb = 3.0 * c[1], qc = c[0];
    if (qa == 0.0) {
        if (qb != 0.0)
            ys.push_back(-qc / qb);
    } else {
        double disc = qb * qb - 4.0 * qa * qc;
        if (disc >= 0.0) {
            double sq = std::sqrt(disc);
            // numerically stable pair of roots
            double q = -0.5 * (qb + (qb >= 0 ? sq : -sq));
            if (q != 0.0) {
                ys.push_back(q / qa);
                ys.push_back(qc / q);
            } else {
                ys.push_back(0.0);
            }
        }
    }
    std::vector<double> xs;
    for (double y : ys)
        if (y > 0.0) {
            double x = std::sqrt(y);
            if (x > lo && x < hi)
                xs.push_back(x);
        }
    std::sort(xs.begin(), xs.end());
    return xs;
}

// Extrema of e(x) = 1 - p(x) on [lo, hi] by scanning p' for sign changes and
// bisecting (used only if the closed-form stationary points are not two).
std::vector<double> stationary_scan(const double c[3], double lo, double hi)
{
    auto dp = [&](double x) { double x2 = x * x; return c[0] + x2 * (3.0 * c[1] + 5.0 * c[2] * x2); };
    std::vector<double> xs;
    const int n = 8192;
    double xprev = lo, dprev = dp(lo);
    for (int i = 1; i <= n; ++i) {
        double x = lo + (hi - lo) * i / n;
        double d = dp(x);
        if ((dprev < 0) != (d < 0)) {
            double a = xprev, b = x, da = dprev;
            for (int it = 0; it < 200; ++it) {
                double mid = 0.5 * (a + b);
                double dm = dp(mid);
                if ((da < 0) == (dm < 0)) { a = mid; da = dm; } else { b = mid; }
            }
            double r = 0.5 * (a + b);
            if (r > lo && r < hi)
                xs.push_back(r);
        }
        xprev = x;
        dprev = d;
    }
    return xs;
}

// Minimax odd quintic for the constant 1 on [lo, hi]. Returns the levelled error.
double remez_quintic(double lo, double hi, double coef[3])
{
    const double kPi = 3.14159265358979323846;
    double ref[4];
    for (int k = 0; k < 4; ++k)
        ref[k] = 0.5 * (lo + hi) - 0.5 * (hi - lo) * std::cos(kPi * k / 3.0);
    double lev = 0.0;
    for (int it = 0; it < 200; ++it) {
        double m[4][5];
        for (int k = 0; k < 4; ++k) {
            double x = ref[k], x2 = x * x;
            m[k][0] = x;
            m[k][1] = x * x2;
            m[k][2] = x * x2 * x2;
            m[k][3] = (k % 2 == 0) ? 1.0 : -1.0;
            m[k][4] = 1.0;
        }
        double y[4];
        if (!solve4(m, y))
            break;
        coef[0] = y[0];
        coef[1] = y[1];
        coef[2] = y[2];
        lev = std::fabs(y[3]);
        std::vector<double> st = stationary(coef, lo, hi);
        if (st.size() != 2)
            st = stationary_scan(coef, lo, hi);
        if (st.size() != 2)
            break;
        double nref[4] = {lo, st[0], st[1], hi};
        double moved = 0.0;
        for (int k = 0; k < 4; ++k)
            moved = std::max(moved, std::fabs(nref[k] - ref[k]));
        for (int k = 0; k < 4; ++k)
            ref[k] = nref[k];
        if (moved <= 1e-15 * hi)
            break;
    }
    double emax = lev;
    std::vector<double> st = stationary(coef, lo, hi);
    emax = std::max(emax, std::fabs(1.0 - peval(coef, lo)));
    emax = std::max(emax, std::fabs(1.0 - peval(coef, hi)));
    for (double x : st)
        emax = std::max(emax, std::fabs(1.0 - peval(coef, x)));
    return emax;
}

} // namespace

int schedule_coeffs(int kind, int iters, double ell0, double delta, double *coef, double *lo_out)
{
    if (iters < 0 || (iters > 0 && !coef))
        return 1;
    if (kind == SVT_SCHED_NS3) {
        double lo = (ell0 > 0.0 && ell0 < 1.0) ? ell0 : 1e-3;
        for (int t = 0; t < iters; ++t) {
            coef[3 * t] = 1.5;
            coef[3 * t + 1] = -0.5;
            coef[3 * t + 2] = 0.0;
            if (lo_out)
                lo_out[t] = lo;
            lo = 1.5 * lo - 0.5 * lo * lo * lo;  // the cubic is increasing on [0, 1]
        }
        return 0;
    }
    if (!(ell0 > 0.0 && ell0 < 1.0) || !(delta >= 0.0))
        return 1;
    double lo = ell0, hi = 1.0;
    for (int t = 0; t < iters; ++t) {
        double c[3];
        if (lo_out)
            lo_out[t] = lo;
        double dhi = hi * (1.0 + delta);
        if (dhi - lo < kSwitchWidth) {
            c[0] = 15.0 / 8.0;
            c[1] = -10.0 / 8.0;
            c[2] = 3.0 / 8.0;
            double vmin = std::min(peval(c, lo), peval(c, dhi));
            double vmax = std::max(peval(c, lo), peval(c, dhi));
            for (double x : stationary(c, lo, dhi)) {
                vmin = std::min(vmin, peval(c, x));
                vmax = std::max(vmax, peval(c, x));
            }
            lo = vmin;
            hi = vmax;
        } else {
            double e = remez_quintic(lo, dhi, c);
            lo = 1.0 - e;
            hi = 1.0 + e;
        }
        coef[3 * t] = c[0];
        coef[3 * t + 1] = c[1];
        coef[3 * t + 2] = c[2];
    }
    return 0;
}

} // namespace svt
