/*
 * glm.h - C ABI of libglm: maximum-likelihood reconstruction of recurrent
 * synaptic connectivity from spike trains with a point-process generalised
 * linear model (Zaytsev, Morrison & Deger, "Reconstruction of recurrent
 * synaptic connectivity of thousands of neurons from simulated spiking
 * activity"), evaluated on a time grid on one NVIDIA GB300 (sm_103a).
 *
 * Problem statement (Sec. 2.1-2.3).  N neurons are recorded for T bins of
 * width dt seconds; S_i[t] in {0, 1} says whether neuron i spiked in bin t
 * (Sec. 2.1: spike trains {t_ik} on [T0, T1]).  With a = exp(-dt / tau):
 *   X_j[0] = 0,  X_j[t] = a X_j[t-1] + S_j[t-1]            filtered trains, Eq. 13
 *   U_i[t] = b_i + sum_j W_ij X_j[t]                       potential, Eq. 3
 *   L_i    = sum_t S_i[t] U_i[t] - dt sum_t exp(U_i[t])    log-likelihood, Eq. 2/5/7
 *   dL_i/dW_ij = sum_t R_i[t] X_j[t],  dL_i/db_i = sum_t R_i[t],
 *   R_i[t] = S_i[t] - dt exp(U_i[t])                       gradient, Eq. 11-12
 * b_i is the paper's baseline J_i0 (base rate c_i = exp(b_i) in 1/s, Eq. 6),
 * W_ij its J_ij (weight of the connection j -> i, gain du = 1), tau the
 * membrane time constant of the exponential kernel (Sec. 2.2).  A spike
 * acts from the next bin on: every connection, the self-connection included,
 * carries a delay of one bin (the paper's d_s = dt, Sec. 2.4 and 3.1).
 * L = sum_i L_i (Eq. 1) and every row is an independent concave problem
 * (Sec. 2.2, App. A).
 *
 * Conventions for every call:
 *   - Return value: GLM_OK (0) on success, a negative GLM_ERR_* on error, a
 *     positive GLM_STATUS_* for a finished call with a noteworthy outcome.
 *     A call that fails validation changes nothing.  glm_strerror() names
 *     every code; glm_last_error() gives a message for the context's last
 *     failure.
 *   - Ownership: the caller owns every buffer it passes and the library
 *     never frees or keeps one.  The context owns its device workspace
 *     (spikes, filtered trains, spike term, partial sums) and frees it in
 *     glm_destroy().
 *   - Memory kinds: parameters named *_dev are device pointers on the
 *     context's device, *_host are host pointers.  Matrices are row-major.
 *   - Streams: work is queued on the stream given to glm_create() (NULL =
 *     the legacy default stream).  A call that writes a *_host output
 *     synchronises that stream before returning; other calls may return
 *     before the device work is finished.
 *   - Thread safety: a context must not be used from two threads at once;
 *     different contexts are independent.
 */
#ifndef GLM_H
#define GLM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define GLM_OK 0
#define GLM_ERR_INVALID_ARG (-1)        /* null pointer, non-positive size, dt/tau not finite and > 0, ... */
#define GLM_ERR_UNSORTED_SPIKES (-2)    /* bins of a row not strictly increasing (two spikes in one bin) */
#define GLM_ERR_SPIKE_OUT_OF_RANGE (-3) /* a bin outside [0, n_bins), or offsets not a valid CSR */
#define GLM_ERR_OOM (-4)                /* device allocation failed or the workspace cap was exceeded */
#define GLM_ERR_CUDA (-5)               /* a CUDA runtime/driver call failed */
#define GLM_ERR_NONFINITE (-6)          /* non-finite W or b, or exp(U) overflowed */
#define GLM_ERR_TIMEOUT (-7)            /* a bounded device-side wait gave up */
#define GLM_ERR_UNSUPPORTED_ARCH (-8)   /* a tensor-core precision was asked for on a GPU other than sm_103 */
#define GLM_ERR_NO_PROBLEM (-9)         /* the call needs glm_set_problem() first */
#define GLM_ERR_UNSUPPORTED (-10)       /* valid request outside what the library implements */

/* ---- precision of the contractions U = b + W X and G = R X^T ----
 * GLM_PREC_F32:  the plain FP32 form.  X (correctly rounded from a
 *                double-float scan) and the rates stored in FP32, SIMT FP32
 *                products on CUDA cores, FP64 sums across tiles; the spike
 *                term sum_t S_i[t] X_j[t] (Eq. 12, the part that does not
 *                depend on W, computed once per problem as Sec. 2.3.3 and
 *                2.6.1 advise) summed from double-float X.
 * GLM_PREC_BF16: tcgen05 tensor cores.  W split into hi + lo BF16 parts, so
 *                that W_hi X + W_lo X keeps W to ~16 significant bits; X held
 *                as X_hi + X_lo BF16 parts (U adds W_hi X_lo) unless
 *                glm_set_x_split(ctx, 0) asks for X_hi alone; the rates
 *                dt*exp(U) stored in BF16; FP32 accumulation in tensor
 *                memory; FP64 sums across tiles.  The spike term is the
 *                tensor-core product S X^T over the same X.
 * GLM_PREC_F16:  as GLM_PREC_BF16 with IEEE half instead of BF16. */
typedef enum { GLM_PREC_F32 = 0, GLM_PREC_BF16 = 1, GLM_PREC_F16 = 2 } glm_prec_t;

/* element types for glm_filter outputs */
typedef enum { GLM_DTYPE_F32 = 0, GLM_DTYPE_BF16 = 1, GLM_DTYPE_F16 = 2 } glm_dtype_t;

typedef struct glm_ctx glm_ctx;

/* Version of the library as major * 10000 + minor * 100 + patch. */
int glm_version(void);

/* Static name of a status code; never NULL. */
const char* glm_strerror(int code);

/* Message describing the last error raised on ctx (empty if none); valid until the next call on ctx. */
const char* glm_last_error(const glm_ctx* ctx);

/* Create a context on CUDA device `device`.
 *   workspace_cap_bytes: upper bound on the device memory the context may hold (0 = no bound);
 *                        exceeding it makes the call that needed more return GLM_ERR_OOM.
 *   cuda_stream:         a cudaStream_t on that device, or NULL for the legacy default stream.
 * On success *out receives the context.  Errors: INVALID_ARG, CUDA. */
int glm_create(glm_ctx** out, int device, size_t workspace_cap_bytes, void* cuda_stream);

/* Release the context and all device memory it owns.  NULL is ignored. */
void glm_destroy(glm_ctx* ctx);

/* Set the recording (Sec. 2.1) and the model constants, then prepare the per-problem caches
 * (steps a0-a2: filtered trains X for the chosen precision and the spike term).
 *   n, n_bins:  neurons and bins, n >= 1, 1 <= n_bins < 2^31.
 *   dt, tau:    bin width and kernel time constant in seconds, both finite and > 0.
 *   offs_host:  int64[n + 1] CSR offsets, offs[0] = 0, non-decreasing.
 *   bins_host:  int32[offs[n]] spike bins; row i is bins[offs[i] .. offs[i+1]), strictly increasing,
 *               each in [0, n_bins).  At most one spike per neuron and bin.
 *   prec:       precision of the contractions (glm_prec_t).
 * The spikes are copied to the device; the host arrays may be freed on return.  Replaces any previous
 * problem.  A recording with the current problem's n, n_bins, spike count, precision, chunking and delay
 * reuses its buffers: its spikes are copied to a second device buffer (allocated by the first such call) and
 * checked there, and replace the current ones only when they pass; otherwise the host checks them.  Either
 * way a recording that fails the check changes nothing and gets the same error and message.
 * Errors: INVALID_ARG, UNSORTED_SPIKES, SPIKE_OUT_OF_RANGE, OOM, CUDA, UNSUPPORTED_ARCH. */
int glm_set_problem(glm_ctx* ctx, int32_t n, int64_t n_bins, double dt, double tau, const int64_t* offs_host,
                    const int32_t* bins_host, glm_prec_t prec);

/* Continuous-time form of the same model (Sec. 2.3, Eq. 7-14): spike times in seconds, off any grid.
 * Every spike reaches every neuron after one uniform delay (Sec. 2.4, Eq. 15 with D_ij = delay), so the
 * potential is U_i(t) = b_i + sum_j W_ij v_j(t), v_j(t) = sum over arrivals e <= t of exp(-(t - e) / tau)
 * (Eq. 3, 11; an arrival counts at its own time), and L_i = sum_k U_i(t_ik) - int exp(U_i) dt over
 * [t_begin, t_end) (Eq. 2, 7).  The library cuts the recording at every distinct arrival and spike time
 * into event columns; the U product runs over the columns, and the integral over each column is the
 * exact one of Eq. 9-10 (its Ei closed form is evaluated by Gauss-Legendre quadrature in exp(-s/tau),
 * see glm_ct_interval), with the matching interval weights of Eq. 14 in the gradient.
 *   n:                 neurons, n >= 1.
 *   t_begin, t_end:    the recording window in seconds, finite, t_begin < t_end.
 *   tau:               kernel time constant in seconds, finite and > 0.
 *   delay:             transmission delay in seconds, finite and >= 0 (0: a spike counts in its own U).
 *   offs_host:         int64[n + 1] CSR offsets, offs[0] = 0, non-decreasing; offs[n] < 2^30.
 *   times_host:        double[offs[n]] spike times; row i strictly increasing, each in [t_begin, t_end).
 *   prec:              GLM_PREC_BF16 or GLM_PREC_F16 (the FP32 form covers the grid only: UNSUPPORTED).
 * Afterwards glm_prepare, glm_spike_term, glm_loglik_grad (dL/dtau included), glm_fit and
 * glm_cross_validate work on the columns as they do on bins, and a chunk length set by glm_set_chunk_bins
 * (in columns) recomputes v chunk by chunk as X on the grid; glm_filter and glm_fit_batch return
 * UNSUPPORTED.  The host arrays may be freed on return.
 * Errors: INVALID_ARG, UNSORTED_SPIKES, SPIKE_OUT_OF_RANGE, OOM, CUDA, UNSUPPORTED, UNSUPPORTED_ARCH. */
int glm_set_problem_ct(glm_ctx* ctx, int32_t n, double t_begin, double t_end, double tau, double delay,
                       const int64_t* offs_host, const double* times_host, glm_prec_t prec);

/* Number of time columns of the current problem: n_bins on the grid, the event columns (distinct
 * arrival and spike times, plus the column starting at t_begin) in continuous time.
 * Errors: INVALID_ARG, NO_PROBLEM. */
int glm_problem_columns(const glm_ctx* ctx, int64_t* n_columns);

/* The two interval integrals of the continuous-time form over one column of length D, for a potential
 * that relaxes as U(s) = b + u exp(-s / tau) (Eq. 8 between events), with b = 0, computed by the same
 * FP32 code as the U-product epilogue:
 *   F = int_0^D exp(u exp(-s / tau)) ds              (= tau (Ei(u) - Ei(u a)), a = exp(-D / tau), Eq. 10)
 *   G = int_0^D exp(-s / tau) exp(u exp(-s / tau)) ds (= tau (e^u - e^{u a}) / u, Eq. 14)
 * Host function, needs no GPU.  Errors: INVALID_ARG (D < 0, tau <= 0, non-finite u, D or tau, NULL
 * outputs). */
int glm_ct_interval(double u, double D, double tau, double* F_host, double* G_host);

/* The explicit tau-derivative of the column integral F above at fixed u, as the dL/dtau epilogue computes
 * it in FP32: dF/dtau = (F - D e^{u a}) / tau = u int_a^1 e^{u rho} (-ln rho) d rho (by parts from the
 * definition of F; quadrature in 1 - rho for columns with 1 - a <= 0.1, the first form otherwise).  Host
 * function, needs no GPU.  Errors: INVALID_ARG (as glm_ct_interval). */
int glm_ct_interval_dtau(double u, double D, double tau, double* dFdtau_host);

/* e^v - 1 for each of n FP32 values, as the plain FP32 form's link epilogue evaluates it (the rate of Eq. 5
 * is e^b (1 + (e^v - 1)) with v = sum_j W_ij X_j): Cody-Waite reduction and a Taylor series in double-float,
 * rounded once, i.e. correctly rounded but for rare near-ties, so that its rounding does not bias the
 * integral of Eq. 7.  Host function, needs no GPU; the device code is the same source.
 * Errors: INVALID_ARG (n < 0, NULL arrays with n > 0). */
int glm_expm1(const float* v_host, int64_t n, float* out_host);

/* ---- per-neuron time constants and delays (Sec. 2.2, Sec. 2.4 Eq. 15) ----
 * The paper's kernel h_i(t) = H(t) exp(-t / tau_i) belongs to the target neuron i, and Eq. 15 shifts every
 * source train S_j by the delay D_ij of the target that receives it.  The rows (targets) are grouped into
 * classes of equal (tau, delay); one context per class holds that class's filtered trains (all N sources,
 * filtered with the class's tau and shifted by its delay) and evaluates and fits only the class's rows.
 * Number the neurons so that each class is a contiguous block of rows. */

/* Delay in bins with which every source train reaches the rows (delay_bins >= 1; 1, the default, is the
 * one-bin delay of the grid recursion X[t] = a X[t-1] + S[t-1]).  Above 1 the filter reads each spike
 * delay_bins - 1 bins later (spikes pushed past the recording drop out); the rows' own spikes, for the
 * spike-time term, stay where they are.  Takes effect at the next glm_set_problem (grid form).
 * Errors: INVALID_ARG (delay_bins < 1). */
int glm_set_source_delay(glm_ctx* ctx, int32_t delay_bins);

/* Self-delay (Sec. 2.4, Eq. 15 with D_ii != D_ij; the paper's own network uses one delay d for every
 * connection and a separate self-delay d_s, Sec. 3.1): each row's own train reaches it after self_bins bins
 * while every other train arrives after the source delay (glm_set_source_delay).  1 <= self_bins <= the
 * source delay (a self-delay equal to it, or 0, the default, leaves the model as it is).  U_i then has the
 * diagonal term W_ii X_i[t + d - d_s], X filtered with the source delay d: the filtered trains extend d - d_s
 * bins past the recording, and the U product, the spike term's diagonal and dL/dW_ii use that shifted row.
 * Takes effect at the next glm_set_problem of a tensor-core grid problem with X stored; glm_set_problem
 * returns UNSUPPORTED for the plain FP32 form or a chunked problem with a self-delay, and glm_loglik_grad
 * does for dL/dtau, as do glm_set_problem_ct and glm_fit_batch.  Errors: INVALID_ARG (self_bins < 0). */
int glm_set_self_delay(glm_ctx* ctx, int32_t self_bins);

/* Restrict evaluations and fits of the current problem to rows [r0, r1) (0 <= r0 < r1 <= n; r0 = 0 with
 * r1 = 0 or n restores all rows).  glm_loglik_grad then forms U, the rates and the gradient for those rows
 * only and returns L_i = 0, dL/dW_i. = 0 and dL/db_i = 0 for the others (L_total sums the range);
 * glm_fit leaves the other rows' W and b as given, with state GLM_ROW_EXCLUDED.  Not with glm_fit_batch.
 * Errors: INVALID_ARG, NO_PROBLEM. */
int glm_set_row_range(glm_ctx* ctx, int32_t r0, int32_t r1);


/* Ward's minimum-variance hierarchical clustering of neurons by their weights (Sec. 3.4.2, Ward 1963): the
 * paper clusters the reconstructed connectivity by outgoing weights (columns of W) and, inside clusters,
 * by incoming weights (rows) to expose the links of a synfire chain.
 *   W_dev:        float[n * n] weights (device, row-major, W[i, j] = weight of j -> i).
 *   by:           0: point k is the column W[:, subset[k]] (outgoing); 1: the row W[subset[k], :] (incoming).
 *   subset_host:  int32[m] neuron indices to cluster, or NULL for all n (m is then n).
 *   Z_host:       double[(m - 1) * 4] the linkage in SciPy's layout: row q = (id_a, id_b, height, size),
 *                 ids < m are the points (positions in the subset), m + q the cluster made by row q,
 *                 id_a < id_b, heights non-decreasing; height = sqrt(2 x the rise in within-cluster sum of
 *                 squares) = the Ward distance.
 * Squared distances in FP64 on the device, then a nearest-neighbour-chain walk with the Lance-Williams
 * update in one block; uses O(m^2 + m n) doubles of temporary device memory and the context's stream
 * (the context needs no problem).  Errors: INVALID_ARG, OOM, CUDA, NONFINITE (the walk did not complete:
 * non-finite weights). */
int glm_ward(glm_ctx* ctx, const float* W_dev, int32_t n, int32_t by, const int32_t* subset_host, int32_t m,
             double* Z_host);

/* Labels 0 .. k-1 of the k clusters left after the first m - k merges of a linkage (clusters numbered by
 * their smallest member).  Host function.  Errors: INVALID_ARG. */
int glm_ward_cut(const double* Z_host, int32_t m, int32_t k, int32_t* labels_host);

/* ---- checks of the library itself (the paper has no counterpart) ----
 * glm_poison_caches: fill every buffer that glm_prepare and glm_loglik_grad recompute (filtered trains,
 * rates, partial sums, spike term, segment carries, column constants) with the byte 0xFF, i.e. NaN in
 * every floating type, and mark the spike term stale.  After glm_prepare the results must be those of a
 * fresh context bit for bit: no kernel reads a value it did not write (padding bins and rows included).
 * Errors: INVALID_ARG, NO_PROBLEM, CUDA.
 * glm_check_wait_limit: run the bounded mbarrier wait of the tensor-core kernels on a barrier nobody
 * arrives on, with limit_seconds in [1e-4, 2].  Returns GLM_ERR_TIMEOUT when the wait gave up and
 * reported it (the expected outcome; the context stays usable), GLM_ERR_CUDA if it did not.  The context
 * needs no problem. */
int glm_poison_caches(glm_ctx* ctx);
int glm_check_wait_limit(glm_ctx* ctx, double limit_seconds);

/* Recompute the per-problem caches (filter scan, spike term) from the device-resident spikes, for a new
 * tau (tau > 0) or, with tau <= 0, the current one.  Errors: NO_PROBLEM, INVALID_ARG, CUDA. */
int glm_prepare(glm_ctx* ctx, double tau);

/* Write the filtered trains X[:, t0 : t0 + t_len] (Eq. 13) of the current problem into X_dev, row-major
 * with leading dimension ldx elements (ldx >= t_len), element type dtype.  Computed afresh by the scan
 * kernel.  Errors: NO_PROBLEM, INVALID_ARG (range outside [0, n_bins), ldx < t_len), CUDA. */
int glm_filter(glm_ctx* ctx, int64_t t0, int64_t t_len, void* X_dev, int64_t ldx, glm_dtype_t dtype);

/* Copy the spike term C_ij = sum_t S_i[t] X_j[t] (n x n, FP64, row-major) and the spike counts
 * q_i (FP64) of the current problem into device buffers; either may be NULL.
 * Errors: NO_PROBLEM, CUDA. */
int glm_spike_term(glm_ctx* ctx, double* C_dev, double* q_dev);

/* Log-likelihood and gradient of the current problem at (W, b) (steps a3-a6, a7):
 *   W_dev: float[n * n], b_dev: float[n]  (inputs, device)
 *   L_rows_dev:   double[n]      L_i                    (or NULL)
 *   L_total_host: double         L = sum_i L_i          (or NULL; synchronises)
 *   G_dev:        double[n * n]  dL_i / dW_ij           (or NULL: the gradient product is skipped)
 *   gb_dev:       double[n]      dL_i / db_i            (or NULL)
 *   gtau_host:    double         dL / dtau              (or NULL; synchronises).  tau enters through
 *                 a = exp(-dt/tau) in the kernel of Eq. 3 (it is not part of theta_i, Sec. 2.2):
 *                 dL/dtau = (a dt / tau^2) sum_{i,t} R_i[t] sum_j W_ij dX_j[t]/da.  In continuous time
 *                 (glm_set_problem_ct) tau also sets each column's integral: dL/dtau = sum over spikes
 *                 of z_i / tau^2 - e^{b_i} sum_m [G_m z_m / tau^2 + dF_m/dtau at fixed u] with z = W dv/dtau
 *                 tau^2 (see glm_ct_interval_dtau).  The first request on a problem also computes its
 *                 W-independent spike part.  Tensor-core precisions only (GLM_ERR_UNSUPPORTED for
 *                 GLM_PREC_F32).
 * Errors: NO_PROBLEM, INVALID_ARG, NONFINITE (exp(U) overflowed; outputs are then undefined), CUDA,
 * TIMEOUT, UNSUPPORTED, OOM. */
int glm_loglik_grad(glm_ctx* ctx, const float* W_dev, const float* b_dev, double* L_rows_dev,
                    double* L_total_host, double* G_dev, double* gb_dev, double* gtau_host);

/* ---- maximum-likelihood fit (Sec. 2.2 separability, Sec. 2.6.3 optimiser and stopping rule) ----
 * Every row i is an independent concave problem in theta_i = (b_i, W_i1..W_in) (App. A).  All rows are
 * fitted together: each iteration evaluates every active row's trial point in one batched evaluation,
 * and each row keeps its own search direction, step and history. */
#define GLM_FIT_LBFGS 0 /* limited-memory BFGS (the paper's optimiser family, Sec. 2.6.3) */
#define GLM_FIT_GA 1    /* plain gradient ascent */

#define GLM_ROW_CONVERGED 0
#define GLM_ROW_MAXITER 1
#define GLM_ROW_STALLED 2
#define GLM_ROW_DEGENERATE 3
#define GLM_ROW_AT_FLOOR 4 /* stopped at the evaluation's resolution: even a steepest-ascent step predicts a
                              gain below gain_floor (|L_i| + q_i), so no further increase can be told apart
                              from the evaluation's rounding (typical of the 16-bit precisions near the
                              optimum, whose L_i carry a relative error of ~1e-7) */
#define GLM_ROW_EXCLUDED 5 /* outside the context's row range (glm_set_row_range): not fitted, W_i and b_i
                              returned as given */

#define GLM_STATUS_NOT_CONVERGED 1 /* some row reached max_iter */
#define GLM_STATUS_STALLED 2       /* some row's line search failed (no increase found) */

typedef struct {
    int32_t method;       /* GLM_FIT_LBFGS (default) or GLM_FIT_GA */
    int32_t m;            /* L-BFGS memory, 1..32 (default 10) */
    int32_t max_iter;     /* iteration cap (default 500) */
    double eta;           /* row stop: |L_i(new) - L_i(old)| / |L_i(old)| < eta (default 1e-10; Sec. 2.6.3) */
    double c1;            /* Armijo sufficient-increase constant (default 1e-4) */
    int32_t max_halvings; /* backtracking steps of one line search (each shrinks the step 2-10x) before
                             the row restarts from the gradient or, without history, stalls (default 40) */
    int32_t warm_start;   /* 0: start at W = 0, b_i = log(q_i / (T dt)); 1: start at the W, b passed in */
    double gain_floor;    /* a row whose predicted gain s |g.d| falls below gain_floor (|L_i| + q_i) during
                             its line search is declared stalled: smaller gains are not resolved by the
                             evaluation.  < 0 (default): 1e-13 for GLM_PREC_F32, 1e-10 for BF16/F16;
                             0 disables the test. */
    double alpha;         /* smooth l1 penalty (Sec. 2.5, Eq. 16-17): maximise L_i - alpha sum_{j != i}
                             sqrt(W_ij^2 + eps); the bias and the self weight are not penalised.  0 (default):
                             plain maximum likelihood */
    double eps;           /* epsilon of the smooth l1 form, > 0 (default 1e-6) */
} glm_fit_opts_t;

typedef struct {
    int32_t iterations;  /* outer iterations */
    int32_t evaluations; /* log-likelihood evaluations (U products), trials included */
    int32_t gradients;   /* gradient products */
    int32_t converged, maxiter, stalled, degenerate, at_floor; /* rows in each final state */
    int32_t excluded;    /* rows outside the row range */
    double L;            /* final log-likelihood sum_i L_i */
    double seconds;      /* wall time of the call */
} glm_fit_report_t;

/* Fill *opts with the defaults above. */
void glm_fit_default_opts(glm_fit_opts_t* opts);

/* Maximum-likelihood W and b of the current problem.
 *   W_dev: float[n * n], b_dev: float[n] (device).  Read when opts->warm_start, always overwritten with
 *          the fit.  Rows with no spike have no finite maximum in b_i: they get b_i = log(1e-3 / s) (the
 *          lower bound of the paper's base-rate box, Sec. 2.6.3), W_i = 0 and state DEGENERATE.
 *   row_status_host: optional int8[n] receiving GLM_ROW_* per row.
 *   report: optional.
 * Returns GLM_OK when every non-degenerate row converged or stopped at the floor, GLM_STATUS_NOT_CONVERGED or GLM_STATUS_STALLED
 * otherwise (the fit is still written), or a negative GLM_ERR_*.  Synchronises the context's stream. */
int glm_fit(glm_ctx* ctx, const glm_fit_opts_t* opts, float* W_dev, float* b_dev, int8_t* row_status_host,
            glm_fit_report_t* report);

/* Fit several independent recordings together (the batched form of glm_fit).  ctxs[p] holds problem p
 * (set with glm_set_problem; uneven n and n_bins are fine); all contexts are on the same device and use
 * the same tensor-core precision (GLM_PREC_BF16 or GLM_PREC_F16).  Every evaluation is one launch of each
 * contraction over the tiles of all problems, and one optimiser iteration for all of them (directions,
 * line-search rounds, gradient, update) is recorded once as a CUDA graph and replayed; a line search that
 * is still open after an iteration's rounds continues in the next iteration.  All work runs on ctxs[0]'s
 * stream.  W_dev[p], b_dev[p]: as for glm_fit; row_status_host and reports: optional arrays of n_prob
 * (row_status_host[p] may be NULL).  n_prob: 1..32.  Returns the worst of the per-problem glm_fit
 * statuses or a negative GLM_ERR_* (INVALID_ARG for mixed devices, precisions or X splits; UNSUPPORTED for
 * GLM_PREC_F32, continuous-time and chunked problems, row ranges and self-delays).  Synchronises ctxs[0]'s stream. */
#define GLM_FIT_BATCH_MAX 32
int glm_fit_batch(glm_ctx* const* ctxs, int32_t n_prob, const glm_fit_opts_t* opts, float* const* W_dev,
                  float* const* b_dev, int8_t* const* row_status_host, glm_fit_report_t* reports);

/* Fit every class: glm_fit on each context in turn (each with its own tau, delay and row range; the row
 * ranges must not overlap), all writing into the one W_dev (n x n) and b_dev (n).  row_status_host
 * (optional, int8[n]) receives each row's state from the context that owns it (GLM_ROW_EXCLUDED for rows
 * in no range); the report sums the classes' counts and times (iterations: the largest).  Returns the
 * most severe status of the classes' fits.  Errors: INVALID_ARG (overlapping ranges, differing n or
 * device), NO_PROBLEM, and those of glm_fit. */
int glm_fit_classes(glm_ctx* const* ctxs, int32_t n_class, const glm_fit_opts_t* opts, float* W_dev, float* b_dev,
                    int8_t* row_status_host, glm_fit_report_t* report);

/* Cross-validation of the l1 penalty (Sec. 2.5) and of the kernel time constant (Sec. 3.2): for every tau in
 * taus and every alpha in alphas, fit W, b on ctx_train (glm_fit with opts and that alpha) and evaluate the
 * log-likelihood of the fit on ctx_valid, a recording of the same neurons over other bins (e.g. the second
 * half of one recording).  taus: n_tau values (> 0), or NULL with n_tau = 1 to keep both problems' tau;
 * alphas: n_alpha values >= 0, fitted in the order given, each fit starting from the previous one (an
 * ascending list keeps every start close).  L_valid_host: optional double[n_tau * n_alpha], index
 * k_tau * n_alpha + k_alpha; best_host: optional int32[2] receiving (k_tau, k_alpha) of the largest
 * validation log-likelihood; W_best_dev (float[n*n]) and b_best_dev (float[n]) receive the fit there.  Both
 * contexts hold problems of the same n and precision on the same device; their tau is left at the last
 * value tried.  Errors: as glm_fit and glm_loglik_grad, INVALID_ARG for mismatched problems. */
int glm_cross_validate(glm_ctx* ctx_train, glm_ctx* ctx_valid, const glm_fit_opts_t* opts, const double* alphas,
                       int32_t n_alpha, const double* taus, int32_t n_tau, double* L_valid_host, int32_t* best_host,
                       float* W_best_dev, float* b_best_dev);

/* Recompute X chunk by chunk instead of storing it, for recordings whose N x n_bins outgrows device memory
 * (hour-long recordings of thousands of neurons).  chunk_bins > 0 (rounded up to a multiple of 4096) applies to the next
 * glm_set_problem of a tensor-core precision: the context then holds X (or X_hi and X_lo) and the rates
 * for chunk_bins bins only, and every evaluation filters, multiplies and reduces one chunk after the other
 * (the filter runs once per chunk and evaluation, so an evaluation costs one filter pass more).  0
 * (default) stores X for the whole recording.  Ignored for GLM_PREC_F32 and when chunk_bins covers the
 * recording.  For glm_set_problem_ct it counts event columns.  Chunked problems cannot be batched
 * (glm_fit_batch). */
int glm_set_chunk_bins(glm_ctx* ctx, int64_t chunk_bins);

/* How the 16-bit grid forms hold X (the filtered trains of Eq. 13), for the next glm_set_problem.  split = 1
 * (default): X = X_hi + X_lo, two 16-bit arrays; U takes three tensor-core products (W_hi X_hi, W_lo X_hi,
 * W_hi X_lo) and the spike term two (S X_hi^T, S X_lo^T), and X keeps ~16 significant bits in BF16 and ~22
 * in F16.  split = 0: X_hi alone, the round-to-nearest 16-bit X; U takes two products (W_hi X, W_lo X),
 * the spike term and E X^T one each, and the filter writes half the bytes of X.  With F16 the single X keeps
 * 11 significant bits, which holds L within ~3e-7 of the FP64 value at N = 1000 (BF16's 8 bits do not: its
 * X rounding moves L by ~6e-6).  Ignored for GLM_PREC_F32 and the continuous-time form (whose columns are
 * always split).  Returns GLM_OK, or INVALID_ARG for split other than 0 or 1. */
int glm_set_x_split(glm_ctx* ctx, int32_t split);

/* ---- autotuner of the gradient product's tile shape ----
 * (no counterpart in the paper.)  Times the gradient product E X^T of the current problem for row tiles of
 * 256 and 128 neurons and 1, 2, 4 and 8 bin splits per SM (the K extent of a tile), and keeps the fastest
 * for the context's later evaluations and fits.  The choice is cached for the process per precision, n,
 * n_bins and GPU, so later contexts of the same shape reuse it without timing.  Results of later calls are
 * reproducible for a given choice; another choice changes the FP32 summation order of the gradient.
 * glm_fit_batch tunes its batched launch the same way, for all its problems at once.  Tensor-core
 * precisions only (GLM_ERR_UNSUPPORTED for GLM_PREC_F32).  Synchronises the context's stream. */
typedef struct {
    int32_t mode;       /* 1: 256-row tiles, 2: 128-row tiles */
    int32_t nsplit;     /* bin splits */
    int32_t cached;     /* 1 if taken from the process cache without timing */
    int32_t candidates; /* candidates timed */
    float best_ms;      /* time of one gradient product with the choice */
} glm_tune_report_t;
int glm_autotune(glm_ctx* ctx, glm_tune_report_t* report);

/* Set the gradient product's tile shape by hand, as one of the autotuner's candidates: mode 1 (256-row
 * tiles) or 2 (128-row tiles), and units_per_sm in {1, 2, 4, 8}, from which the bin splits follow
 * (written to *nsplit_out when not NULL).  Applies to the context's later evaluations and fits until the next
 * glm_set_problem or glm_autotune.  Every candidate computes the same product; they differ in the FP32
 * summation order of the gradient only.  Errors: INVALID_ARG, NO_PROBLEM, UNSUPPORTED (GLM_PREC_F32). */
int glm_set_grad_tile(glm_ctx* ctx, int32_t mode, int32_t units_per_sm, int32_t* nsplit_out);

/* ---- classification of reconstructed weights (Sec. 3.1 GMM, Sec. 3.3 k-means, Table 2, Eq. 20) ---- */
#define GLM_CLASSIFY_GMM 0    /* 3-component Gaussian mixture by EM, started from 3-means (default) */
#define GLM_CLASSIFY_KMEANS 1 /* 3-means (Lloyd) */

typedef struct {
    int32_t method;   /* GLM_CLASSIFY_GMM or GLM_CLASSIFY_KMEANS */
    int32_t max_iter; /* iteration cap of each stage (default 1000) */
    double tol;       /* GMM stop: relative change of the mixture log-likelihood (default 1e-12) */
} glm_classify_opts_t;

typedef struct {
    double centers[3];   /* cluster centres / component means, ascending: inhibitory, absent, excitatory */
    double weights[3];   /* GMM mixing weights (0 for k-means) */
    double variances[3]; /* GMM variances (0 for k-means) */
    double loglik;       /* final GMM log-likelihood */
    int32_t iterations;  /* iterations of the last stage */
    int64_t errors;      /* misclassified off-diagonal pairs (needs truth) */
    double mer;          /* errors / (n (n - 1)), the denominator of Eq. 20 */
    double mer_n2;       /* errors / n^2, the denominator of Table 2 */
    int64_t fp[3], fn[3], nd[3]; /* per class (index 0 inhibitory, 1 absent, 2 excitatory): false
                                    positives, false negatives, and false positives that contradict
                                    Dale's law for the presynaptic type (needs types) */
} glm_classify_report_t;

/* Classify the off-diagonal weights of W_host (n x n, row-major, W[i][j] = weight of j -> i; host) into
 * labels_out (n x n int8, host): -1 inhibitory, 0 absent, +1 excitatory; the diagonal is set to 0.
 *   opts:  NULL for the defaults.
 *   truth: optional n x n int8 ground-truth labels (host) for the error report; types: optional int8[n]
 *          (+1 excitatory, -1 inhibitory presynaptic neuron) for the Dale's-law count.
 *   report: optional.
 * Runs on the host; needs no context.  Errors: INVALID_ARG (n < 2, null W or labels, bad options),
 * NONFINITE (a non-finite weight). */
int glm_classify(const double* W_host, int32_t n, const glm_classify_opts_t* opts, int8_t* labels_out,
                 const int8_t* truth_host, const int8_t* types_host, glm_classify_report_t* report);

/* ---- allocation-free log-likelihood ----
 * The paper has no counterpart to this call; it exists for callers that may not allocate device memory:
 * processes whose device memory belongs to another allocator (a framework's caching pool, a pre-reserved
 * arena) and loops that must not call cudaMalloc after start-up.  It needs no context and allocates
 * nothing itself: its temporary storage is one fixed array of GLM_NOALLOC_SCRATCH_BYTES in device memory,
 * part of the library's device code, which a GPU holds from the moment that code is loaded on it until the
 * process exits.  With CUDA's default lazy module loading that moment is the first call of this function
 * on the device (not the loading of the library): the first call commits the 16 MiB and fails with
 * GLM_ERR_CUDA if the device has no room left.  Make that first call at start-up, before another allocator
 * reserves the device's memory, or run the process with CUDA_MODULE_LOADING=EAGER; later calls commit
 * nothing.  The array's device address is looked up on that first call and kept for the process: it stays
 * valid for the life of the device's primary context (after cudaDeviceReset, do not call this function
 * again in the same process).
 *
 * Computes the per-row log-likelihood of the plain FP32 form (the same quantity as glm_loglik_grad's
 * L_rows for a GLM_PREC_F32 problem) from caller buffers, all device pointers on the current device:
 *   X_dev:  float [n][ldx], the filtered trains X[:, 0 : n_bins] (e.g. from glm_filter), ldx >= n_bins
 *   C_dev:  double [n][n], the spike term (e.g. from glm_spike_term);  q_dev: double [n], spike counts
 *   W_dev:  float [n][n];  b_dev: float [n]
 *   L_rows_dev: double [n] output.  A non-finite exp(U) or input shows up as a non-finite L_i.
 *   cuda_stream: the stream to queue the work on (NULL = legacy default stream); the call does not wait.
 * Needs n * (ceil(n_bins / 128) + 1) * 8 bytes <= GLM_NOALLOC_SCRATCH_BYTES, else returns
 * GLM_ERR_SCRATCH_TOO_SMALL without doing anything.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) once for that device: make that first call outside any stream
 * capture.  All calls share the one array, so calls whose work overlaps on the GPU (two streams, two host
 * threads) race; serialise them.  Errors: INVALID_ARG, SCRATCH_TOO_SMALL, CUDA. */
#define GLM_NOALLOC_SCRATCH_BYTES (16u << 20)
#define GLM_ERR_SCRATCH_TOO_SMALL (-11)
int glm_loglik_noalloc(int32_t n, int64_t n_bins, double dt, const float* X_dev, int64_t ldx, const double* C_dev,
                       const double* q_dev, const float* W_dev, const float* b_dev, double* L_rows_dev,
                       void* cuda_stream);

/* ---- tracing ----
 * While profiling is enabled, every kernel group the context launches (filter_scan, carry, spike_term,
 * u_epilogue, grad, reduce, ...) is bracketed by CUDA events recorded on the context's stream.
 * glm_profile_read() synchronises that stream and writes, for up to max_entries groups, the group name
 * (NUL-terminated, 32 bytes per entry in names), the number of launches and the summed device time in
 * milliseconds since profiling was last enabled; it returns the number of entries written (>= 0) or a
 * negative GLM_ERR_*.  glm_profile_enable(ctx, 1) also resets the totals. */
int glm_profile_enable(glm_ctx* ctx, int enable);
int glm_profile_read(glm_ctx* ctx, int max_entries, char* names, int64_t* launches, double* ms);

/* Number of CUDA kernels the context has launched since it was created (a running counter). */
int64_t glm_launch_count(const glm_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* GLM_H */
