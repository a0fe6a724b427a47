/*
 * FP64 one-sided Jacobi (Hestenes) SVD -- TEST INFRASTRUCTURE ONLY.
 *
 * Part of the oracle for singular value soft-thresholding. Only the tests, the
 * package smoke check and the benchmark's CPU-baseline leg may load this code;
 * the GPU library never does, and this file shares nothing with it.
 *
 * The SVT target (Eq. 1) is A_tau = U max(Sigma - tau I, 0) V^T, defined from the
 * singular value decomposition A = U Sigma V^T (Section 2). This file supplies that
 * decomposition by the textbook one-sided Jacobi method:
 *
 *   W <- A (m x n, m >= n), V <- I_n.
 *   Repeat sweeps over all column pairs (i, j):
 *     alpha = w_i.w_i, beta = w_j.w_j, gamma = w_i.w_j;
 *     if |gamma| > eps * sqrt(alpha * beta), rotate columns i, j of W and of V by
 *     the plane rotation that makes w_i.w_j = 0.
 *   Stop after a sweep in which no pair needed a rotation.
 *   sigma_i = ||w_i||, u_i = w_i / sigma_i (zero column when sigma_i = 0).
 *
 * The pair order is the round-robin (circle) tournament: each round is a set of
 * n/2 disjoint pairs, processed in parallel with OpenMP. The tolerance is
 * eps = m * 2^-53 unless the caller passes another one.
 *
 * Layout: the caller's A, U and V are row-major; W and V are kept column-major
 * internally so that column operations are contiguous.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* One plane rotation of columns p < q of W (length m) and V (length n).
 * Returns 1 if a rotation was applied. */
static int rotate_pair(double *W, double *V, int64_t m, int64_t n, int64_t p, int64_t q,
                       double eps)
{
    double *wp = W + p * m, *wq = W + q * m;
    double alpha = 0.0, beta = 0.0, gamma = 0.0;
    for (int64_t r = 0; r < m; ++r) {
        alpha += wp[r] * wp[r];
        beta += wq[r] * wq[r];
        gamma += wp[r] * wq[r];
    }
    if (gamma == 0.0 || fabs(gamma) <= eps * sqrt(alpha * beta))
        return 0;
    /* zeta = (beta - alpha) / (2 gamma); t = tan(theta) is the smaller root of
     * t^2 + 2 zeta t - 1 = 0, so that the rotated pair is orthogonal. */
    double zeta = (beta - alpha) / (2.0 * gamma);
    double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
    double c = 1.0 / sqrt(1.0 + t * t);
    double s = c * t;
    for (int64_t r = 0; r < m; ++r) {
        double a = wp[r], b = wq[r];
        wp[r] = c * a - s * b;
        wq[r] = s * a + c * b;
    }
    double *vp = V + p * n, *vq = V + q * n;
    for (int64_t r = 0; r < n; ++r) {
        double a = vp[r], b = vq[r];
        vp[r] = c * a - s * b;
        vq[r] = s * a + c * b;
    }
    return 1;
}

/*
 * oracle_jacobi_svd: thin SVD of a row-major m x n FP64 matrix with m >= n.
 *   A      in : m x n row-major.
 *   sigma  out: n singular values, sorted descending.
 *   U      out: m x n row-major, columns u_i (zero where sigma_i = 0).
 *   V      out: n x n row-major, columns v_i.
 *   eps       : orthogonality tolerance; <= 0 selects m * 2^-53.
 *   max_sweeps: sweep limit (the result is returned even if not converged).
 *   nthreads  : OpenMP threads (<= 0 keeps the runtime default).
 *   max_rounds: if > 0, stop after this many tournament rounds in total (a
 *               bounded sample of the work, for timing; the result is then not
 *               converged).
 *   sweeps_out: number of sweeps run; off_out: max |gamma|/sqrt(alpha beta) over
 *               all pairs at exit.
 * Returns 0 when converged, 1 when a limit was hit, -1 on bad arguments.
 */
int oracle_jacobi_svd(int64_t m, int64_t n, const double *A, double *sigma, double *U,
                      double *V, double eps, int max_sweeps, int max_rounds, int nthreads,
                      int *sweeps_out, double *off_out)
{
    if (m < n || n <= 0 || !A || !sigma || !U || !V)
        return -1;
    if (eps <= 0.0)
        eps = (double)m * ldexp(1.0, -53);
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    double *W = (double *)malloc(sizeof(double) * (size_t)(m * n));
    double *Vc = (double *)calloc((size_t)(n * n), sizeof(double));
    int64_t np2 = n + (n & 1); /* players in the tournament; index n is a bye */
    int64_t *ring = (int64_t *)malloc(sizeof(int64_t) * (size_t)np2);
    if (!W || !Vc || !ring) {
        free(W); free(Vc); free(ring);
        return -1;
    }
    for (int64_t r = 0; r < m; ++r)
        for (int64_t c = 0; c < n; ++c)
            W[c * m + r] = A[r * n + c];
    for (int64_t c = 0; c < n; ++c)
        Vc[c * n + c] = 1.0;

    int sweeps = 0, converged = 0, limited = 0;
    int64_t rounds_done = 0;
    while (sweeps < max_sweeps && !converged && !limited) {
        ++sweeps;
        int rotations = 0;
        for (int64_t i = 0; i < np2; ++i)
            ring[i] = i;
        for (int64_t round = 0; round < np2 - 1; ++round) {
            /* Pair k of this round: ring[k] with ring[np2 - 1 - k]. */
            int round_rot = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : round_rot)
            for (int64_t k = 0; k < np2 / 2; ++k) {
                int64_t p = ring[k], q = ring[np2 - 1 - k];
                if (p >= n || q >= n)
                    continue;
                if (p > q) { int64_t t = p; p = q; q = t; }
                round_rot += rotate_pair(W, Vc, m, n, p, q, eps);
            }
            rotations += round_rot;
            /* Circle method: keep ring[0], rotate the rest by one place. */
            int64_t last = ring[np2 - 1];
            for (int64_t i = np2 - 1; i > 1; --i)
                ring[i] = ring[i - 1];
            ring[1] = last;
            if (max_rounds > 0 && ++rounds_done >= max_rounds) {
                limited = 1;
                break;
            }
        }
        if (rotations == 0 && !limited)
            converged = 1;
    }

    /* Largest remaining normalised off-diagonal value (diagnostic). */
    double off = 0.0;
    if (off_out) {
#pragma omp parallel for schedule(dynamic, 8) reduction(max : off)
        for (int64_t p = 0; p < n; ++p) {
            for (int64_t q = p + 1; q < n; ++q) {
                double a = 0, b = 0, g = 0;
                const double *wp = W + p * m, *wq = W + q * m;
                for (int64_t r = 0; r < m; ++r) {
                    a += wp[r] * wp[r]; b += wq[r] * wq[r]; g += wp[r] * wq[r];
                }
                double d = (a > 0 && b > 0) ? fabs(g) / sqrt(a * b) : 0.0;
                if (d > off) off = d;
            }
        }
        *off_out = off;
    }

    /* sigma_i = ||w_i||; order descending (stable insertion sort of indices). */
    double *nrm = (double *)malloc(sizeof(double) * (size_t)n);
    int64_t *ord = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    for (int64_t c = 0; c < n; ++c) {
        double s = 0.0;
        for (int64_t r = 0; r < m; ++r)
            s += W[c * m + r] * W[c * m + r];
        nrm[c] = sqrt(s);
        ord[c] = c;
    }
    for (int64_t i = 1; i < n; ++i) {
        int64_t key = ord[i], j = i - 1;
        while (j >= 0 && nrm[ord[j]] < nrm[key]) {
            ord[j + 1] = ord[j];
            --j;
        }
        ord[j + 1] = key;
    }
    for (int64_t k = 0; k < n; ++k) {
        int64_t c = ord[k];
        double s = nrm[c];
        sigma[k] = s;
        for (int64_t r = 0; r < m; ++r)
            U[r * n + k] = (s > 0.0) ? W[c * m + r] / s : 0.0;
        for (int64_t r = 0; r < n; ++r)
            V[r * n + k] = Vc[c * n + r];
    }
    free(nrm); free(ord);
    free(W); free(Vc); free(ring);
    if (sweeps_out)
        *sweeps_out = sweeps;
    return converged ? 0 : 1;
}

/* Number of OpenMP threads a parallel region would use (1 without OpenMP). */
int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
