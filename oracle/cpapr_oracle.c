/*
 * CP-APR MU oracle: a plain, slow, FP64 CPU implementation of what the GPU
 * path computes, written from the paper (arXiv 2307.03276, "Analyzing the
 * Performance Portability of Tensor Decomposition").
 *
 * TEST INFRASTRUCTURE ONLY.  It is loaded by the tests, by the smoke check
 * and by the benchmark's CPU-baseline leg, never by the CUDA library, and it
 * shares no code, header or table with it.
 *
 * Conventions: N modes, mode m has I_m rows.  Coordinates are 0-based and
 * passed mode-major: idx[m * nnz + j] is the mode-m coordinate of nonzero j.
 * Factor matrices are row-major I_m x R.  Nonzeros are visited in the order
 * given (no sorting, no blocking, no fusion).
 *
 * Every row sum of Phi, of MTTKRP and the log-likelihood sum use Neumaier's
 * compensated summation (A. Neumaier, ZAMM 54, 1974), so that the oracle's
 * own rounding error stays near one unit in the last place even for rows
 * with millions of terms.
 *
 * Readings of points the paper leaves open:
 *  - epsilon, kappa, kappa_tol are parameters (defaults 1e-10, 0.01, 1e-10);
 *  - S (the inadmissible-zero shift of Algorithm 1, step B <- (A+S)Lambda)
 *    follows Chi and Kolda: S(i,r) = kappa when k > 1, A(i,r) < kappa_tol
 *    and the previous outer iteration's Phi(i,r) > 1, else 0;
 *  - the KKT check runs after Phi and before B <- B * Phi and stops the inner
 *    loop when max_{i,r} |min(B(i,r), 1 - Phi(i,r))| < tol;
 *  - the outer loop stops when every mode passed its KKT check at the first
 *    inner iteration, else after max_outer iterations;
 *  - a column with lambda_r = 0 keeps its A(:,r) unchanged;
 *  - LL = sum_nz x log(m) - sum over all entries of the model, i.e. the
 *    Poisson log-likelihood without the constant sum log(x!).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_E_ARG 1
#define ORACLE_E_RANGE 2
#define ORACLE_E_NOMEM 4

/* Neumaier summation step: s + c carries the running sum.  Once the sum is
 * infinite (a log(0) term of the log-likelihood) the compensation stops. */
static void nsum_add(double *s, double *c, double x)
{
    double t = *s + x;
    if (!isfinite(t)) {
        *s = t;
        return;
    }
    if (fabs(*s) >= fabs(x))
        *c += (*s - t) + x;
    else
        *c += (x - t) + *s;
    *s = t;
}

static int check_coords(int N, const int64_t *dims, int64_t nnz, const int64_t *idx)
{
    for (int m = 0; m < N; ++m)
        for (int64_t j = 0; j < nnz; ++j)
            if (idx[(int64_t)m * nnz + j] < 0 || idx[(int64_t)m * nnz + j] >= dims[m])
                return ORACLE_E_RANGE;
    return ORACLE_OK;
}

/*
 * Phi^(n) by Algorithm 2, evaluated one nonzero at a time as Algorithm 3
 * does (one nonzero j at a time):
 *   pi_j[r] = prod_{m != n} A^(m)[i_m(j), r]          (row j of Pi^T)
 *   s_j     = sum_r B[i_n(j), r] * pi_j[r]            (entry of B Pi)
 *   v_j     = x_j / max(s_j, eps)                     (X_(n) ./ max(B Pi, eps))
 *   Phi[i_n(j), r] += v_j * pi_j[r]                   (... times Pi^T)
 * Zero entries of X contribute nothing, so only nonzeros are visited.
 * With unit_denominator != 0 the division is skipped (v_j = x_j): that is
 * the MTTKRP of the paper's Experiment 8, M = X_(n) (Khatri-Rao of A^(m))
 * (element-wise product, scale, add).
 */
int oracle_phi(int N, const int64_t *dims, int64_t nnz, const int64_t *idx, const double *vals,
               int R, const double *const *A, const double *B, int n, double eps,
               int unit_denominator, double *Phi)
{
    if (N < 2 || R < 1 || n < 0 || n >= N || nnz < 0)
        return ORACLE_E_ARG;
    if (check_coords(N, dims, nnz, idx))
        return ORACLE_E_RANGE;
    int64_t In = dims[n];
    double *comp = calloc((size_t)In * R + 1, sizeof(double));
    double *pi = malloc(sizeof(double) * R);
    if (!comp || !pi) {
        free(comp);
        free(pi);
        return ORACLE_E_NOMEM;
    }
    memset(Phi, 0, sizeof(double) * (size_t)In * R);
    for (int64_t j = 0; j < nnz; ++j) {
        int64_t i = idx[(int64_t)n * nnz + j];
        for (int r = 0; r < R; ++r)
            pi[r] = 1.0;
        for (int m = 0; m < N; ++m) {
            if (m == n)
                continue;
            const double *row = A[m] + idx[(int64_t)m * nnz + j] * R;
            for (int r = 0; r < R; ++r)
                pi[r] *= row[r];
        }
        double v = vals[j];
        if (!unit_denominator) {
            double s = 0.0;
            for (int r = 0; r < R; ++r)
                s += B[i * R + r] * pi[r];
            v = vals[j] / (s > eps ? s : eps);
        }
        for (int r = 0; r < R; ++r)
            nsum_add(&Phi[i * R + r], &comp[i * R + r], v * pi[r]);
    }
    for (int64_t e = 0; e < In * R; ++e)
        Phi[e] += comp[e];
    free(comp);
    free(pi);
    return ORACLE_OK;
}

/*
 * The same Phi^(n) (or MTTKRP) on several host threads, for timing the CPU
 * baseline on all of a machine's cores.  Thread t owns the rows
 * [row0, row1) of Phi^(n), a range holding about nnz / nthreads nonzeros;
 * it visits every nonzero in the given order and evaluates those whose
 * mode-n coordinate falls in its rows exactly as oracle_phi does.  Each row
 * is therefore summed by one thread, term by term in the same order and with
 * the same Neumaier compensation as oracle_phi: the result is bit-for-bit
 * oracle_phi's, with no per-thread copies of Phi to merge.
 */
struct phi_rows {
    int N;
    const int64_t *dims;
    int64_t nnz;
    const int64_t *idx;
    const double *vals;
    int R;
    const double *const *A;
    const double *B;
    int n;
    double eps;
    int unit_denominator;
    int64_t row0, row1;  /* rows of Phi this thread owns */
    double *Phi, *comp;  /* I_n x R values and compensations (shared, disjoint rows) */
};

static void *phi_rows_run(void *arg)
{
    struct phi_rows *c = (struct phi_rows *)arg;
    const int R = c->R, n = c->n;
    double pi[256];  /* R <= 256 (checked by the caller) */
    for (int64_t j = 0; j < c->nnz; ++j) {
        int64_t i = c->idx[(int64_t)n * c->nnz + j];
        if (i < c->row0 || i >= c->row1)
            continue;
        for (int r = 0; r < R; ++r)
            pi[r] = 1.0;
        for (int m = 0; m < c->N; ++m) {
            if (m == n)
                continue;
            const double *row = c->A[m] + c->idx[(int64_t)m * c->nnz + j] * R;
            for (int r = 0; r < R; ++r)
                pi[r] *= row[r];
        }
        double v = c->vals[j];
        if (!c->unit_denominator) {
            double s = 0.0;
            for (int r = 0; r < R; ++r)
                s += c->B[i * R + r] * pi[r];
            v = c->vals[j] / (s > c->eps ? s : c->eps);
        }
        for (int r = 0; r < R; ++r)
            nsum_add(&c->Phi[i * R + r], &c->comp[i * R + r], v * pi[r]);
    }
    for (int64_t e = c->row0 * R; e < c->row1 * R; ++e)
        c->Phi[e] += c->comp[e];
    return NULL;
}

int oracle_phi_threads(int N, const int64_t *dims, int64_t nnz, const int64_t *idx, const double *vals,
                       int R, const double *const *A, const double *B, int n, double eps,
                       int unit_denominator, double *Phi, int nthreads)
{
    if (N < 2 || R < 1 || R > 256 || n < 0 || n >= N || nnz < 0 || nthreads < 1)
        return ORACLE_E_ARG;
    if (check_coords(N, dims, nnz, idx))
        return ORACLE_E_RANGE;
    const int64_t In = dims[n];
    struct phi_rows *ch = calloc((size_t)nthreads, sizeof(struct phi_rows));
    pthread_t *th = calloc((size_t)nthreads, sizeof(pthread_t));
    char *running = calloc((size_t)nthreads, 1);
    int64_t *count = calloc((size_t)In + 1, sizeof(int64_t));
    double *comp = calloc((size_t)In * R + 1, sizeof(double));
    if (!ch || !th || !running || !count || !comp) {
        free(ch);
        free(th);
        free(running);
        free(count);
        free(comp);
        return ORACLE_E_NOMEM;
    }
    memset(Phi, 0, sizeof(double) * (size_t)In * R);
    /* row ranges of about nnz / nthreads nonzeros each */
    for (int64_t j = 0; j < nnz; ++j)
        count[idx[(int64_t)n * nnz + j]] += 1;
    int64_t row = 0, seen = 0;
    for (int t = 0; t < nthreads; ++t) {
        struct phi_rows *c = &ch[t];
        c->N = N;
        c->dims = dims;
        c->nnz = nnz;
        c->idx = idx;
        c->vals = vals;
        c->R = R;
        c->A = A;
        c->B = B;
        c->n = n;
        c->eps = eps;
        c->unit_denominator = unit_denominator;
        c->Phi = Phi;
        c->comp = comp;
        c->row0 = row;
        const int64_t target = nnz * (t + 1) / nthreads;
        while (row < In && (seen < target || t == nthreads - 1))
            seen += count[row++];
        c->row1 = row;
    }
    for (int t = 1; t < nthreads; ++t)
        running[t] = pthread_create(&th[t], NULL, phi_rows_run, &ch[t]) == 0;
    for (int t = 0; t < nthreads; ++t)
        if (!running[t])
            phi_rows_run(&ch[t]);  /* range 0, and any range no thread could take */
    for (int t = 1; t < nthreads; ++t)
        if (running[t])
            pthread_join(th[t], NULL);
    free(ch);
    free(th);
    free(running);
    free(count);
    free(comp);
    return ORACLE_OK;
}

/*
 * Model value at nonzero j: m_j = sum_r lambda_r prod_m A^(m)[i_m(j), r]
 * (the Kruskal model [lambda; A^(1) .. A^(N)] of Algorithm 1's input).
 */
static double model_value(int N, int64_t nnz, const int64_t *idx, int64_t j, int R,
                          const double *lambda, const double *const *A)
{
    double mj = 0.0;
    for (int r = 0; r < R; ++r) {
        double p = lambda[r];
        for (int m = 0; m < N; ++m)
            p *= A[m][idx[(int64_t)m * nnz + j] * R + r];
        mj += p;
    }
    return mj;
}

/*
 * Poisson log-likelihood of the model, without the constant sum log(x!):
 *   LL = sum_nz x_j log(m_j) - sum_{all entries} M
 * and sum over all entries of M = sum_r lambda_r prod_m (sum_i A^(m)[i, r]).
 * A nonzero with m_j = 0 gives -inf.
 */
double oracle_loglik(int N, const int64_t *dims, int64_t nnz, const int64_t *idx, const double *vals,
                     int R, const double *lambda, const double *const *A)
{
    double s = 0.0, c = 0.0;
    for (int64_t j = 0; j < nnz; ++j) {
        double mj = model_value(N, nnz, idx, j, R, lambda, A);
        nsum_add(&s, &c, vals[j] * log(mj));
    }
    double total = 0.0, tc = 0.0;
    for (int r = 0; r < R; ++r) {
        double p = lambda[r];
        for (int m = 0; m < N; ++m) {
            double cs = 0.0, cc = 0.0;
            for (int64_t i = 0; i < dims[m]; ++i)
                nsum_add(&cs, &cc, A[m][i * R + r]);
            p *= cs + cc;
        }
        nsum_add(&total, &tc, p);
    }
    return (s + c) - (total + tc);
}

/* max_{i,r} |min(B(i,r), 1 - Phi(i,r))| : the KKT violation of one mode. */
static double kkt_violation(int64_t In, int R, const double *B, const double *Phi)
{
    double v = 0.0;
    for (int64_t e = 0; e < In * R; ++e) {
        double a = B[e] < 1.0 - Phi[e] ? B[e] : 1.0 - Phi[e];
        a = fabs(a);
        if (a > v)
            v = a;
    }
    return v;
}

/*
 * Algorithm 1 (CP-APR MU), in the paper's order:
 *   for k = 1..k_max, for n = 1..N:
 *     B <- (A^(n) + S) Lambda
 *     Pi <- Khatri-Rao of the other factors (formed per nonzero inside Phi)
 *     for l = 1..l_max:  Phi <- Algorithm 2;  [KKT check];  B <- B * Phi
 *     lambda <- e^T B;  A^(n) <- B Lambda^{-1}
 * lambda (R) and the factors (A[m], I_m x R) are updated in place.
 * Traces (may be NULL): ll_trace[k] = LL after outer iteration k,
 * kkt_trace[k] = largest last-checked violation over modes in iteration k,
 * inner_trace[k*N+n] = inner iterations run for mode n in iteration k.
 */
int oracle_mu_solve(int N, const int64_t *dims, int64_t nnz, const int64_t *idx, const double *vals,
                    int R, double *lambda, double *const *A, double tol, int max_outer, int max_inner,
                    double eps, double kappa, double kappa_tol, int *outer_done, int *total_inner,
                    int *converged, double *ll_trace, double *kkt_trace, int *inner_trace)
{
    if (N < 2 || R < 1 || max_outer < 0 || max_inner < 1 || nnz < 0)
        return ORACLE_E_ARG;
    if (check_coords(N, dims, nnz, idx))
        return ORACLE_E_RANGE;
    int64_t Imax = 0;
    for (int m = 0; m < N; ++m)
        if (dims[m] > Imax)
            Imax = dims[m];
    double *B = malloc(sizeof(double) * (size_t)Imax * R + 8);
    double **Phi = calloc(N, sizeof(double *));
    if (!B || !Phi) {
        free(B);
        free(Phi);
        return ORACLE_E_NOMEM;
    }
    for (int m = 0; m < N; ++m) {
        Phi[m] = calloc((size_t)dims[m] * R + 1, sizeof(double));
        if (!Phi[m]) {
            for (int q = 0; q < m; ++q)
                free(Phi[q]);
            free(Phi);
            free(B);
            return ORACLE_E_NOMEM;
        }
    }
    int k_done = 0, inner_sum = 0, conv = 0;
    for (int k = 1; k <= max_outer; ++k) {
        int all_first = 1;
        double kkt_k = 0.0;
        for (int n = 0; n < N; ++n) {
            int64_t In = dims[n];
            /* B <- (A^(n) + S) Lambda */
            for (int64_t i = 0; i < In; ++i)
                for (int r = 0; r < R; ++r) {
                    double a = A[n][i * R + r];
                    double s = (k > 1 && a < kappa_tol && Phi[n][i * R + r] > 1.0) ? kappa : 0.0;
                    B[i * R + r] = (a + s) * lambda[r];
                }
            int l, passed = 0;
            double viol = 0.0;
            for (l = 1; l <= max_inner; ++l) {
                oracle_phi(N, dims, nnz, idx, vals, R, (const double *const *)A, B, n, eps, 0, Phi[n]);
                viol = kkt_violation(In, R, B, Phi[n]);
                if (viol < tol) {
                    passed = 1;
                    break;
                }
                for (int64_t e = 0; e < In * R; ++e)
                    B[e] *= Phi[n][e];
            }
            int used = passed ? l : max_inner;
            inner_sum += used;
            if (inner_trace)
                inner_trace[(k - 1) * N + n] = used;
            if (!(passed && l == 1))
                all_first = 0;
            if (viol > kkt_k)
                kkt_k = viol;
            /* lambda <- e^T B ;  A^(n) <- B Lambda^{-1} */
            for (int r = 0; r < R; ++r) {
                double cs = 0.0, cc = 0.0;
                for (int64_t i = 0; i < In; ++i)
                    nsum_add(&cs, &cc, B[i * R + r]);
                lambda[r] = cs + cc;
            }
            for (int64_t i = 0; i < In; ++i)
                for (int r = 0; r < R; ++r)
                    if (lambda[r] > 0.0)
                        A[n][i * R + r] = B[i * R + r] / lambda[r];
        }
        k_done = k;
        if (kkt_trace)
            kkt_trace[k - 1] = kkt_k;
        if (ll_trace)
            ll_trace[k - 1] = oracle_loglik(N, dims, nnz, idx, vals, R, lambda, (const double *const *)A);
        if (all_first) {
            conv = 1;
            break;
        }
    }
    if (outer_done)
        *outer_done = k_done;
    if (total_inner)
        *total_inner = inner_sum;
    if (converged)
        *converged = conv;
    for (int m = 0; m < N; ++m)
        free(Phi[m]);
    free(Phi);
    free(B);
    return ORACLE_OK;
}

/* --------------------------------------------------------------------------
 * Random initial model.  SplitMix64 (Steele, Lea, Flood, OOPSLA 2014),
 * written from its published definition: state += golden; output =
 * mix(state).  Entry e of factor m is U(0,1) from draw e of the sub-stream
 * whose base is output (200 + m) of a generator seeded with `seed`.  Each
 * column is then scaled to sum to one and lambda_r collects the product of
 * the original column sums.
 * ------------------------------------------------------------------------ */
static uint64_t sm64_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static uint64_t sm64_draw(uint64_t base, uint64_t i)
{
    return sm64_mix(base + (i + 1) * 0x9E3779B97F4A7C15ULL);
}

int oracle_init_random(int N, const int64_t *dims, int R, uint64_t seed, double *lambda, double *const *A)
{
    if (N < 2 || R < 1)
        return ORACLE_E_ARG;
    for (int r = 0; r < R; ++r)
        lambda[r] = 1.0;
    for (int m = 0; m < N; ++m) {
        uint64_t base = sm64_draw(seed, (uint64_t)(200 + m));
        for (int64_t e = 0; e < dims[m] * R; ++e)
            A[m][e] = (double)(sm64_draw(base, (uint64_t)e) >> 11) * 0x1.0p-53;
        for (int r = 0; r < R; ++r) {
            double cs = 0.0, cc = 0.0;
            for (int64_t i = 0; i < dims[m]; ++i)
                nsum_add(&cs, &cc, A[m][i * R + r]);
            cs += cc;
            lambda[r] *= cs;
            if (cs > 0.0)
                for (int64_t i = 0; i < dims[m]; ++i)
                    A[m][i * R + r] /= cs;
        }
    }
    return ORACLE_OK;
}
