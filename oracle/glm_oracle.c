/*
 * FP64 oracle for the grid point-process GLM of Zaytsev, Morrison & Deger
 * (connectivity reconstruction from spikes).  TEST INFRASTRUCTURE ONLY: it is
 * the slow, plain definition that the CUDA library is checked against.  Only
 * the test suite, the smoke check and the benchmark's CPU-baseline leg may
 * load it.  It shares no code, header or table with the CUDA library.
 *
 * Model on a grid of T bins of width dt, spike counts S_j[t] (at most one per
 * bin in the data used here), a = exp(-dt/tau):
 *   X_j[0] = 0,  X_j[t] = a X_j[t-1] + S_j[t-1]                 Eq. 13 (v_ij)
 *   U_i[t] = b_i + sum_j W_ij X_j[t]                            Eq. 3
 *   lambda_i[t] = exp(U_i[t])                                   Eq. 5, du = 1
 *   L_i = sum_t S_i[t] U_i[t] - dt sum_t exp(U_i[t])            Eq. 2 / Eq. 7
 *   dL_i/dW_ij = sum_t R_i[t] X_j[t],  dL_i/db_i = sum_t R_i[t],
 *     R_i[t] = S_i[t] - dt exp(U_i[t])                          Eq. 11-12
 *   dL/dtau = (da/dtau) sum_{i,t} R_i[t] sum_j W_ij Y_j[t],
 *     Y_j = dX_j/da:  Y_j[0] = 0,  Y_j[t] = a Y_j[t-1] + X_j[t-1],  da/dtau = a dt / tau^2
 * The one-bin delay (a spike in bin s first acts in bin s+1, self included)
 * reads the paper's delays d and d_s = dt (Sec. 2.4, Eq. 15; Sec. 3.1) onto
 * the grid.  The integral of the rate is the rectangle rule on the grid.
 *
 * The fit follows Sec. 2.6.3: each row i is an independent concave problem
 * (separability, Sec. 2.2), maximised by limited-memory BFGS; we add a
 * backtracking Armijo line search and stop on |dL_i| / |L_i| < eta.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC glm_oracle.c -lm
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OR_OK = 0, OR_EINVAL = -1, OR_ENOMEM = -2 };
enum { FIT_CONVERGED = 0, FIT_MAXITER = 1, FIT_STALLED = 2, FIT_DEGENERATE = 3 };

static int check_spikes(int32_t n, int64_t T, const int64_t* offs, const int32_t* bins) {
    if (n <= 0 || T <= 0 || !offs) return OR_EINVAL;
    if (offs[0] != 0) return OR_EINVAL;
    for (int32_t i = 0; i < n; ++i) {
        if (offs[i + 1] < offs[i]) return OR_EINVAL;
        for (int64_t k = offs[i]; k < offs[i + 1]; ++k) {
            if (bins[k] < 0 || bins[k] >= T) return OR_EINVAL;
            if (k > offs[i] && bins[k] <= bins[k - 1]) return OR_EINVAL;
        }
    }
    return OR_OK;
}

static int set_threads(int32_t n_threads) {
#ifdef _OPENMP
    return n_threads > 0 ? n_threads : omp_get_max_threads();
#else
    (void)n_threads;
    return 1;
#endif
}

/* X (row-major n x T): the filtered spike trains, Eq. 13 on the grid. */
int oracle_filter(int32_t n, int64_t T, double dt, double tau, const int64_t* offs, const int32_t* bins,
                  double* X, int32_t n_threads) {
    if (check_spikes(n, T, offs, bins) || !(dt > 0) || !(tau > 0) || !X) return OR_EINVAL;
    const double a = exp(-dt / tau);
    const int nt = set_threads(n_threads);
#pragma omp parallel for schedule(static) num_threads(nt)
    for (int32_t j = 0; j < n; ++j) {
        int64_t k = offs[j];
        double x = 0.0;
        for (int64_t t = 0; t < T; ++t) {
            X[(size_t)j * T + t] = x;
            double s = 0.0;
            while (k < offs[j + 1] && bins[k] == t) {
                s += 1.0;
                ++k;
            }
            x = a * x + s;
        }
    }
    return OR_OK;
}

/*
 * Streaming evaluation for a list of rows, without storing X: for each bin t
 * the current X[t] and Y[t] vectors of all n neurons are kept, the listed rows
 * accumulate their terms, then X and Y advance one bin.
 *   L[r]          = L_i                         (i = rows[r])
 *   G[r*n + j]    = dL_i / dW_ij                (optional)
 *   gb[r]         = dL_i / db_i                 (optional)
 *   gtau[r]       = row i's share of dL/dtau    (optional)
 */
int oracle_eval_rows(int32_t n, int64_t T, double dt, double tau, const int64_t* offs, const int32_t* bins,
                     const double* W, const double* b, int32_t n_rows, const int32_t* rows, double* L, double* G,
                     double* gb, double* gtau, int32_t n_threads) {
    if (check_spikes(n, T, offs, bins) || !(dt > 0) || !(tau > 0) || !W || !b || n_rows <= 0 || !rows || !L)
        return OR_EINVAL;
    for (int32_t r = 0; r < n_rows; ++r)
        if (rows[r] < 0 || rows[r] >= n) return OR_EINVAL;
    const double a = exp(-dt / tau);
    const int64_t q = offs[n];
    /* spikes of the whole network ordered by bin (counting sort) */
    int64_t* toffs = (int64_t*)calloc((size_t)T + 1, sizeof(int64_t));
    int32_t* tneur = (int32_t*)malloc(sizeof(int32_t) * (size_t)(q > 0 ? q : 1));
    if (!toffs || !tneur) {
        free(toffs);
        free(tneur);
        return OR_ENOMEM;
    }
    for (int64_t k = 0; k < q; ++k) toffs[bins[k] + 1]++;
    for (int64_t t = 0; t < T; ++t) toffs[t + 1] += toffs[t];
    {
        int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)T);
        memcpy(fill, toffs, sizeof(int64_t) * (size_t)T);
        for (int32_t j = 0; j < n; ++j)
            for (int64_t k = offs[j]; k < offs[j + 1]; ++k) tneur[fill[bins[k]]++] = j;
        free(fill);
    }
    int nt = set_threads(n_threads);
    if (nt > n_rows) nt = n_rows;
    int failed = 0;
#pragma omp parallel num_threads(nt)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        const int32_t r0 = (int32_t)(((int64_t)n_rows * tid) / nt);
        const int32_t r1 = (int32_t)(((int64_t)n_rows * (tid + 1)) / nt);
        const int32_t nr = r1 - r0;
        double* x = (double*)calloc((size_t)n, sizeof(double));
        double* y = (double*)calloc((size_t)n, sizeof(double));
        double* acc_L = (double*)calloc((size_t)nr, sizeof(double));
        double* acc_gb = (double*)calloc((size_t)nr, sizeof(double));
        double* acc_gt = (double*)calloc((size_t)nr, sizeof(double));
        double* acc_G = G ? (double*)calloc((size_t)nr * n, sizeof(double)) : NULL;
        int64_t* cur = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nr > 0 ? nr : 1));
        if (!x || !y || !acc_L || !acc_gb || !acc_gt || (G && !acc_G) || !cur) {
#pragma omp atomic write
            failed = 1;
        } else {
            for (int32_t r = 0; r < nr; ++r) cur[r] = offs[rows[r0 + r]];
            for (int64_t t = 0; t < T; ++t) {
                for (int32_t r = 0; r < nr; ++r) {
                    const int32_t i = rows[r0 + r];
                    const double* Wi = W + (size_t)i * n;
                    double u = b[i], z = 0.0;
                    for (int32_t j = 0; j < n; ++j) {
                        u += Wi[j] * x[j];
                        z += Wi[j] * y[j];
                    }
                    double s = 0.0;
                    if (cur[r] < offs[i + 1] && bins[cur[r]] == t) {
                        s = 1.0;
                        cur[r]++;
                    }
                    const double e = exp(u);
                    acc_L[r] += s * u - dt * e;
                    const double rr = s - dt * e;
                    acc_gb[r] += rr;
                    acc_gt[r] += rr * z;
                    if (acc_G) {
                        double* Gr = acc_G + (size_t)r * n;
                        for (int32_t j = 0; j < n; ++j) Gr[j] += rr * x[j];
                    }
                }
                /* advance one bin: Y[t+1] = a Y[t] + X[t], then X[t+1] = a X[t] + S[t] */
                for (int32_t j = 0; j < n; ++j) {
                    y[j] = a * y[j] + x[j];
                    x[j] = a * x[j];
                }
                for (int64_t k = toffs[t]; k < toffs[t + 1]; ++k) x[tneur[k]] += 1.0;
            }
            const double dadtau = a * dt / (tau * tau);
            for (int32_t r = 0; r < nr; ++r) {
                L[r0 + r] = acc_L[r];
                if (gb) gb[r0 + r] = acc_gb[r];
                if (gtau) gtau[r0 + r] = dadtau * acc_gt[r];
                if (G) memcpy(G + (size_t)(r0 + r) * n, acc_G + (size_t)r * n, sizeof(double) * (size_t)n);
            }
        }
        free(x);
        free(y);
        free(acc_L);
        free(acc_gb);
        free(acc_gt);
        free(acc_G);
        free(cur);
    }
    free(toffs);
    free(tneur);
    return failed ? OR_ENOMEM : OR_OK;
}

/* ----------------------------------------------------------------------------
 * Per-row fit.  theta = (b_i, W_i1..W_in).  The objective handed to the
 * minimiser is f = -L_i, or with the smooth l1 penalty of Sec. 2.5 (Eq. 16
 * with the epsilon-l1 form of Eq. 17) f = -L_i + alpha sum_{j != i}
 * sqrt(W_ij^2 + eps); the bias and the self weight are not penalised.
 * -------------------------------------------------------------------------- */
typedef struct {
    int32_t n;
    int64_t T;
    double dt;
    const double* X; /* n x T */
    const int32_t* sp; /* spike bins of this row */
    int64_t q;
    double* U;        /* scratch, T */
    int32_t row;      /* i, for the self weight */
    double alpha, eps;
} row_ctx;

/* f = -L_i(theta) (+ penalty); if g != NULL also g = grad f */
static double row_eval(const row_ctx* c, const double* theta, double* g) {
    const int32_t n = c->n;
    const int64_t T = c->T;
    double* U = c->U;
    for (int64_t t = 0; t < T; ++t) U[t] = theta[0];
    for (int32_t j = 0; j < n; ++j) {
        const double w = theta[1 + j];
        if (w == 0.0) continue;
        const double* Xj = c->X + (size_t)j * T;
        for (int64_t t = 0; t < T; ++t) U[t] += w * Xj[t];
    }
    double spk = 0.0, integ = 0.0;
    for (int64_t k = 0; k < c->q; ++k) spk += U[c->sp[k]];
    for (int64_t t = 0; t < T; ++t) {
        const double e = exp(U[t]);
        integ += e;
        U[t] = -c->dt * e; /* U now holds R without the spike term */
    }
    const double L = spk - c->dt * integ;
    if (g) {
        for (int64_t k = 0; k < c->q; ++k) U[c->sp[k]] += 1.0; /* R = S - dt e^U */
        double gb = 0.0;
        for (int64_t t = 0; t < T; ++t) gb += U[t];
        g[0] = -gb;
        for (int32_t j = 0; j < n; ++j) {
            const double* Xj = c->X + (size_t)j * T;
            double s = 0.0;
            for (int64_t t = 0; t < T; ++t) s += U[t] * Xj[t];
            g[1 + j] = -s;
        }
    }
    double pen = 0.0;
    if (c->alpha > 0.0) {
        for (int32_t j = 0; j < n; ++j) {
            if (j == c->row) continue;
            const double w = theta[1 + j], r = sqrt(w * w + c->eps);
            pen += r;
            if (g) g[1 + j] += c->alpha * w / r;
        }
    }
    return -L + c->alpha * pen;
}

static double dot(const double* a, const double* b, int32_t d) {
    double s = 0.0;
    for (int32_t k = 0; k < d; ++k) s += a[k] * b[k];
    return s;
}

/*
 * method 0: L-BFGS with memory m (two-loop recursion, Liu & Nocedal 1989);
 * method 1: plain gradient ascent.  Both use a backtracking Armijo search
 * (sufficient-increase constant c1, step halving).  Rows with no spike have
 * no finite maximum of b_i: they are reported DEGENERATE with
 * b_i = log(1e-3 / s), the lower bound of the paper's base-rate box, W_i = 0.
 */
int oracle_fit(int32_t n, int64_t T, double dt, double tau, const int64_t* offs, const int32_t* bins,
               int32_t method, int32_t m, int32_t max_iter, double eta, double c1, int32_t max_halvings,
               double alpha, double eps, double* W, double* b, int32_t* iters, int32_t* status, int32_t n_threads,
               int32_t n_rows, const int32_t* rows) {
    /* rows (n_rows of them), when given: fit only these rows (each row is its own problem, Sec. 2.2);
       W, b, iters and status are then indexed by position in the list */
    if (check_spikes(n, T, offs, bins) || !(dt > 0) || !(tau > 0) || !W || !b || !iters || !status) return OR_EINVAL;
    if (rows) {
        if (n_rows < 1) return OR_EINVAL;
        for (int32_t r = 0; r < n_rows; ++r)
            if (rows[r] < 0 || rows[r] >= n) return OR_EINVAL;
    } else {
        n_rows = n;
    }
    if (!(alpha >= 0) || !(eps > 0)) return OR_EINVAL;
    if (m < 1 || m > 64 || max_iter < 0 || !(eta >= 0) || !(c1 > 0 && c1 < 1) || max_halvings < 1)
        return OR_EINVAL;
    double* X = (double*)malloc(sizeof(double) * (size_t)n * (size_t)T);
    if (!X) return OR_ENOMEM;
    oracle_filter(n, T, dt, tau, offs, bins, X, n_threads);
    const int nt = set_threads(n_threads);
    const int32_t d = n + 1;
    int failed = 0;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
    for (int32_t r = 0; r < n_rows; ++r) {
        const int32_t i = rows ? rows[r] : r;
        const int64_t q = offs[i + 1] - offs[i];
        if (q == 0) {
            b[r] = log(1e-3);
            for (int32_t j = 0; j < n; ++j) W[(size_t)r * n + j] = 0.0;
            iters[r] = 0;
            status[r] = FIT_DEGENERATE;
            continue;
        }
        double* mem = (double*)malloc(sizeof(double) * ((size_t)T + (size_t)d * (6 + 2 * (size_t)m) + (size_t)m));
        if (!mem) {
#pragma omp atomic write
            failed = 1;
            continue;
        }
        row_ctx c = {n, T, dt, X, bins + offs[i], q, mem, i, alpha, eps};
        double* x = mem + T;
        double* g = x + d;
        double* dir = g + d;
        double* xt = dir + d;
        double* gt = xt + d;
        double* qv = gt + d;
        double* S = qv + d;              /* m x d */
        double* Y = S + (size_t)m * d;   /* m x d */
        double* rho = Y + (size_t)m * d; /* m */
        int32_t hn = 0, hstart = 0;      /* ring buffer of (s, y) pairs */
        for (int32_t k = 0; k < d; ++k) x[k] = 0.0;
        x[0] = log((double)q / ((double)T * dt)); /* maximiser of L_i at W_i = 0 */
        double f = row_eval(&c, x, g);
        int32_t it = 0, st = FIT_MAXITER;
        double ga_step = 0.0;
        while (it < max_iter) {
            /* search direction */
            if (method == 0 && hn > 0) {
                double alpha_h[64];
                for (int32_t k = 0; k < d; ++k) qv[k] = g[k];
                for (int32_t h = hn - 1; h >= 0; --h) {
                    const int32_t s = (hstart + h) % m;
                    alpha_h[h] = rho[s] * dot(S + (size_t)s * d, qv, d);
                    for (int32_t k = 0; k < d; ++k) qv[k] -= alpha_h[h] * Y[(size_t)s * d + k];
                }
                const int32_t last = (hstart + hn - 1) % m;
                const double gamma = dot(S + (size_t)last * d, Y + (size_t)last * d, d) /
                                     dot(Y + (size_t)last * d, Y + (size_t)last * d, d);
                for (int32_t k = 0; k < d; ++k) qv[k] *= gamma;
                for (int32_t h = 0; h < hn; ++h) {
                    const int32_t s = (hstart + h) % m;
                    const double beta = rho[s] * dot(Y + (size_t)s * d, qv, d);
                    for (int32_t k = 0; k < d; ++k) qv[k] += (alpha_h[h] - beta) * S[(size_t)s * d + k];
                }
                for (int32_t k = 0; k < d; ++k) dir[k] = -qv[k];
            } else {
                for (int32_t k = 0; k < d; ++k) dir[k] = -g[k];
            }
            double gd = dot(g, dir, d);
            if (!(gd < 0)) { /* not a descent direction: restart from the gradient */
                hn = 0;
                for (int32_t k = 0; k < d; ++k) dir[k] = -g[k];
                gd = dot(g, dir, d);
            }
            if (gd == 0.0) {
                st = FIT_CONVERGED;
                break;
            }
            const double gnorm = sqrt(dot(g, g, d));
            double step;
            if (method == 0)
                step = hn > 0 ? 1.0 : fmin(1.0, 1.0 / gnorm);
            else
                step = ga_step > 0 ? 2.0 * ga_step : fmin(1.0, 1.0 / gnorm);
            int accepted = 0;
            double ft = 0.0;
            for (int32_t h = 0; h < max_halvings; ++h) {
                for (int32_t k = 0; k < d; ++k) xt[k] = x[k] + step * dir[k];
                ft = row_eval(&c, xt, NULL);
                if (isfinite(ft) && ft <= f + c1 * step * gd) {
                    accepted = 1;
                    break;
                }
                step *= 0.5;
            }
            if (!accepted) {
                st = FIT_STALLED;
                break;
            }
            ga_step = step;
            ft = row_eval(&c, xt, gt);
            /* curvature pair */
            {
                const int32_t s = (hn < m) ? (hstart + hn) % m : hstart;
                double* sv = S + (size_t)s * d;
                double* yv = Y + (size_t)s * d;
                for (int32_t k = 0; k < d; ++k) {
                    sv[k] = xt[k] - x[k];
                    yv[k] = gt[k] - g[k];
                }
                const double sy = dot(sv, yv, d);
                if (sy > 1e-300) {
                    rho[s] = 1.0 / sy;
                    if (hn < m)
                        hn++;
                    else
                        hstart = (hstart + 1) % m;
                }
            }
            const double rel = fabs(ft - f) / fmax(fabs(f), 1e-300);
            for (int32_t k = 0; k < d; ++k) {
                x[k] = xt[k];
                g[k] = gt[k];
            }
            f = ft;
            ++it;
            if (rel < eta) {
                st = FIT_CONVERGED;
                break;
            }
        }
        b[r] = x[0];
        for (int32_t j = 0; j < n; ++j) W[(size_t)r * n + j] = x[1 + j];
        iters[r] = it;
        status[r] = st;
        free(mem);
    }
    free(X);
    return failed ? OR_ENOMEM : OR_OK;
}
