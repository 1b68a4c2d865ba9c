/*
 * Oracle: plain FP64 CPU Lanczos iteration for resistance distance.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library calls, links or
 * includes this file; only the tests, the smoke check and the benchmark's CPU
 * baseline use it. It shares no code with the CUDA path.
 *
 * What it computes (paper: Section 3, Algorithm 3 and the estimator of
 * Eq. (approx_formula)): for an undirected, connected, weighted graph with
 * W_uv = w_uv > 0, degrees d_u = sum_v w_uv (Section 2.1, generalised to
 * weights), normalised adjacency Ahat = D^{-1/2} W D^{-1/2} (Section 2.2),
 *
 *   v_0 = 0, v_1 = (e_s/sqrt(d_s) - e_t/sqrt(d_t)) / sqrt(1/d_s + 1/d_t), beta_1 = 0
 *   for i = 1..k:  u = Ahat v_i - beta_i v_{i-1};  alpha_i = <u, v_i>;
 *                  u = u - alpha_i v_i;  beta_{i+1} = ||u||;  v_{i+1} = u / beta_{i+1}
 *   rhat_k = (1/d_s + 1/d_t) * e_1^T (I - T_k)^{-1} e_1,
 *
 * with T_k the k-by-k tridiagonal matrix with diagonal alpha_1..alpha_k and
 * off-diagonal beta_2..beta_k. The small system (I - T_k) x = e_1 is solved
 * from scratch after every step by Gaussian elimination without pivoting on
 * the tridiagonal matrix (the Thomas algorithm); I - T_k is symmetric positive
 * definite because the eigenvalues of T_k lie in [lambda_min(Ahat),
 * lambda_2(Ahat)] (proof of Lemma lz_quadratic_err), so no pivoting is needed.
 *
 * Readings of points the paper leaves open:
 *  - breakdown (beta_{i+1} = 0 up to rounding, i.e. the Krylov space is
 *    exhausted): stop; T_i is then exact and rhat_i is the answer.
 *  - the oracle's own stop rule, for "run to convergence": stop after step k
 *    when |rhat_k - rhat_{k-1}| <= stop_tol * rhat_k (stop_tol = 0: run to k_max).
 *  - s == t returns 0 without iterating.
 *
 * The potential of Section 6.3 (the one Algorithm 5 starts from),
 *   phi = sqrt(1/d_s + 1/d_t) * D^{-1/2} V_k (I - T_k)^{-1} e_1,
 * is formed from the stored basis V_k.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* Degrees d_u = sum of the weights of row u (1 per entry when w == NULL). */
void orc_degrees(int64_t n, const int64_t *row_ptr, const float *w, double *deg)
{
    for (int64_t u = 0; u < n; ++u) {
        double d = 0.0;
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e)
            d += w ? (double)w[e] : 1.0;
        deg[u] = d;
    }
}

/* e_1^T (I - T)^{-1} e_1 and, optionally, the whole solution x of (I - T) x = e_1,
 * for the k-by-k tridiagonal T with diagonal a[0..k-1] and off-diagonal b[1..k-1]
 * (b[j] couples rows j-1 and j). Thomas algorithm: forward elimination, then
 * back substitution. Returns NAN if a pivot is not positive. */
static double thomas_e1(int k, const double *a, const double *b, double *x_out, double *work)
{
    /* work: c' (k), d' (k) */
    double *cp = work, *dp = work + k;
    double diag = 1.0 - a[0];
    if (!(diag > 0.0)) return NAN;
    cp[0] = (k > 1) ? (-b[1]) / diag : 0.0;
    dp[0] = 1.0 / diag;
    for (int j = 1; j < k; ++j) {
        double lower = -b[j];
        double m = (1.0 - a[j]) - lower * cp[j - 1];
        if (!(m > 0.0)) return NAN;
        cp[j] = (j + 1 < k) ? (-b[j + 1]) / m : 0.0;
        dp[j] = (0.0 - lower * dp[j - 1]) / m;
    }
    double xj = dp[k - 1];
    if (x_out) x_out[k - 1] = xj;
    for (int j = k - 2; j >= 0; --j) {
        xj = dp[j] - cp[j] * xj;
        if (x_out) x_out[j] = xj;
    }
    return xj; /* x[0] */
}

/* One pair. Returns the number of steps k performed (0 if s == t).
 * r_hist[j]   (optional, length k_max) : rhat after step j+1
 * alpha[j]    (optional, length k_max) : alpha_{j+1}
 * beta[j]     (optional, length k_max+1): beta_{j+1} (beta[0] = beta_1 = 0)
 * V           (optional, n x (k_max+1), column j = v_{j+1}) : the Lanczos basis
 * phi         (optional, length n) : potential of Algorithm 5 from V_k; needs V.
 * *r_out : final rhat. */
int orc_lanczos_pair(int64_t n, const int64_t *row_ptr, const int32_t *col, const float *w,
                     const double *deg, int32_t s, int32_t t, int k_max, double stop_tol,
                     double *r_out, double *r_hist, double *alpha, double *beta, double *V, double *phi)
{
    if (s == t) {
        *r_out = 0.0;
        if (phi) memset(phi, 0, sizeof(double) * (size_t)n);
        return 0;
    }
    double *vprev = calloc((size_t)n, sizeof(double));
    double *vcur = calloc((size_t)n, sizeof(double));
    double *u = calloc((size_t)n, sizeof(double));
    double *isd = malloc(sizeof(double) * (size_t)n);
    double *a = malloc(sizeof(double) * (size_t)(k_max + 1));
    double *b = malloc(sizeof(double) * (size_t)(k_max + 2));
    double *work = malloc(sizeof(double) * 2 * (size_t)(k_max + 1));
    for (int64_t i = 0; i < n; ++i) isd[i] = 1.0 / sqrt(deg[i]);

    const double bnorm2 = 1.0 / deg[s] + 1.0 / deg[t];
    const double bnorm = sqrt(bnorm2);
    vcur[s] = isd[s] / bnorm;
    vcur[t] = -isd[t] / bnorm;
    b[0] = 0.0; /* beta_1 */
    if (V) memcpy(V, vcur, sizeof(double) * (size_t)n);

    double r_prev = 0.0, r_k = 0.0;
    int k = 0;
    for (int i = 0; i < k_max; ++i) {
        /* u = Ahat v_i - beta_i v_{i-1} */
        for (int64_t x = 0; x < n; ++x) {
            double acc = 0.0;
            for (int64_t e = row_ptr[x]; e < row_ptr[x + 1]; ++e) {
                double wv = w ? (double)w[e] : 1.0;
                acc += wv * isd[x] * isd[col[e]] * vcur[col[e]];
            }
            u[x] = acc - b[i] * vprev[x];
        }
        double al = 0.0;
        for (int64_t x = 0; x < n; ++x) al += u[x] * vcur[x];
        for (int64_t x = 0; x < n; ++x) u[x] -= al * vcur[x];
        double nb = 0.0;
        for (int64_t x = 0; x < n; ++x) nb += u[x] * u[x];
        nb = sqrt(nb);
        a[i] = al;
        b[i + 1] = nb;
        k = i + 1;
        if (alpha) alpha[i] = al;
        if (beta) { beta[i] = b[i]; beta[i + 1] = nb; }
        r_k = bnorm2 * thomas_e1(k, a, b, NULL, work);
        if (r_hist) r_hist[i] = r_k;
        /* breakdown: the Krylov space is invariant, T_k is exact */
        if (nb <= 1e-13 * (fabs(al) + b[i]) || !(r_k == r_k)) break;
        for (int64_t x = 0; x < n; ++x) {
            double nv = u[x] / nb;
            vprev[x] = vcur[x];
            vcur[x] = nv;
        }
        if (V && i + 1 < k_max + 1) memcpy(V + (size_t)(i + 1) * (size_t)n, vcur, sizeof(double) * (size_t)n);
        if (stop_tol > 0.0 && i > 0 && fabs(r_k - r_prev) <= stop_tol * fabs(r_k)) break;
        r_prev = r_k;
    }
    *r_out = r_k;
    if (phi && V) {
        double *z = malloc(sizeof(double) * (size_t)k);
        thomas_e1(k, a, b, z, work);
        for (int64_t x = 0; x < n; ++x) {
            double acc = 0.0;
            for (int j = 0; j < k; ++j) acc += V[(size_t)j * (size_t)n + (size_t)x] * z[j];
            phi[x] = bnorm * isd[x] * acc;
        }
        free(z);
    }
    free(vprev); free(vcur); free(u); free(isd); free(a); free(b); free(work);
    return k;
}

/* Many pairs, one pair per OpenMP thread (threads <= 0: the OpenMP default).
 * r_out[p], k_out[p] per pair. Returns the number of threads used. */
int orc_lanczos_batch(int64_t n, const int64_t *row_ptr, const int32_t *col, const float *w,
                      const int32_t *s, const int32_t *t, int64_t npairs, int k_max, double stop_tol,
                      int threads, double *r_out, int32_t *k_out)
{
    double *deg = malloc(sizeof(double) * (size_t)n);
    orc_degrees(n, row_ptr, w, deg);
    int used = 1;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel
    {
#pragma omp single
        used = omp_get_num_threads();
#pragma omp for schedule(dynamic, 1)
        for (int64_t p = 0; p < npairs; ++p)
            k_out[p] = orc_lanczos_pair(n, row_ptr, col, w, deg, s[p], t[p], k_max, stop_tol, &r_out[p],
                                        NULL, NULL, NULL, NULL, NULL);
    }
#else
    (void)threads;
    for (int64_t p = 0; p < npairs; ++p)
        k_out[p] = orc_lanczos_pair(n, row_ptr, col, w, deg, s[p], t[p], k_max, stop_tol, &r_out[p],
                                    NULL, NULL, NULL, NULL, NULL);
#endif
    free(deg);
    return used;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
