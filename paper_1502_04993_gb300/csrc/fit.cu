// glm_fit: maximum-likelihood W and b for every row at once.
//
// Each row i is an independent concave problem in theta_i = (b_i, W_i1..W_in) (Sec. 2.2, App. A); the
// paper maximises each with L-BFGS(-B) and stops on the fractional change of the objective (Sec. 2.6.3).
// Here all rows advance together: one batched evaluation (the U product for every row) serves every row's
// trial point, while each row keeps its own direction, step length, Armijo test and curvature history.
// The optimiser state lives on the device in FP64 (one block per row for the vector work); the host only
// sequences the kernels and reads two counters per line-search round.
//
// With f_i = -L_i and g_i = grad f_i:
//   direction   d_i = -H_i g_i   (L-BFGS two-loop recursion, memory m; d_i = -g_i for gradient ascent or
//                                 when d_i is not a descent direction)
//   trial       theta_i + s_i d_i, s_i = 1 (first step min(1, 1/|g_i|)), shrunk until
//               f_i(trial) <= f_i + c1 s_i g_i.d_i  (Armijo).  Each shrink moves s to the minimiser of the
//               quadratic through f_i, g_i.d_i and f_i(trial), kept within [0.1 s, 0.5 s] (0.1 s after a
//               non-finite trial).  A row whose predicted gain s |g_i.d_i| drops below the gain floor, or
//               that used up its backtracking steps, restarts from -g_i with an empty history if it had
//               one, and is stalled otherwise.
//   stop        |L_i(new) - L_i(old)| / |L_i(old)| < eta
#include <cuda_runtime.h>
#include <type_traits>
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include <chrono>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <vector>

#include "glm_internal.h"

namespace glm {

namespace {

constexpr int FT = 256;  // threads per row block
constexpr int ACTIVE = -1;

__device__ double block_sum(double v, double* sh) {
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];  // fixed order: deterministic
    return s;
}

struct FitState {
    int32_t n, d, m, method;
    double* theta;   // [n][d]
    double* g;       // [n][d]   gradient of -L_i
    double* dir;     // [n][d]
    double* S;       // [m][n][d]
    double* Y;       // [m][n][d]
    double* rho;     // [m][n]
    double* Lcur;    // [n]
    double* step;    // [n]
    double* gd;      // [n]
    double* gastep;  // [n]
    int32_t* status; // [n]  ACTIVE or GLM_ROW_*
    int32_t* pend;   // [n]  1 while the line search of this iteration is open
    int32_t* acc;    // [n]  1 if the step of this iteration was accepted
    int32_t* halv;   // [n]
    int32_t* hn;     // [n]  stored curvature pairs
    int32_t* hs;     // [n]  ring start
    int32_t* iters;  // [n]
    int* counters;   // [4]  active rows, open line searches, rows stopped in this round, rows to evaluate
    const double* qd; // [n]  spike counts
    double floor;     // smallest predicted gain s |g.d| worth testing, relative to |L_i| + q_i
    double alpha, eps; // smooth l1 penalty alpha sum_{j != i} sqrt(W_ij^2 + eps) (Sec. 2.5); alpha = 0: none
    double* pen;       // [n]  penalty sum at each row's last trial point
};

// d/dW of the penalty for theta index k >= 1 (W_i,k-1); the self weight is not penalised
__device__ __forceinline__ double pen_grad(const FitState& F, int32_t i, int k, double w) {
    return (F.alpha > 0.0 && k - 1 != i) ? F.alpha * w / sqrt(w * w + F.eps) : 0.0;
}

// Rows outside [r0, r1) (a row range) keep the caller's W_i and b_i and are not fitted.
__global__ void fit_init_kernel(FitState F, double span, const double* __restrict__ qd, int warm,
                                const float* __restrict__ W, const float* __restrict__ b, int32_t r0, int32_t r1) {
    const int32_t i = blockIdx.x;
    double* th = F.theta + (int64_t)i * F.d;
    const double q = qd[i];
    const bool excl = i < r0 || i >= r1;
    const bool degen = !excl && q == 0.0;
    const bool keep = warm || excl;
    for (int k = threadIdx.x; k < F.d; k += blockDim.x) {
        double v;
        if (k == 0)
            v = degen ? log(1e-3) : (keep ? (double)b[i] : log(q / span));
        else
            v = (degen || !keep) ? 0.0 : (double)W[(int64_t)i * F.n + (k - 1)];
        th[k] = v;
    }
    if (threadIdx.x == 0) {
        F.status[i] = excl ? GLM_ROW_EXCLUDED : degen ? GLM_ROW_DEGENERATE : ACTIVE;
        F.hn[i] = 0;
        F.hs[i] = 0;
        F.iters[i] = 0;
        F.pend[i] = 0;
        F.acc[i] = 0;
        F.gastep[i] = 0.0;
    }
}

// trial point in FP32 for the evaluator: theta + s d for rows with an open or accepted step, theta otherwise
__device__ __forceinline__ void fit_trial_body(const FitState& F, int32_t i, float* __restrict__ W,
                                               float* __restrict__ b) {
    __shared__ double shp[32];
    const bool move = F.status[i] == ACTIVE && (F.pend[i] || F.acc[i]);
    const double s = move ? F.step[i] : 0.0;
    const double* th = F.theta + (int64_t)i * F.d;
    const double* dr = F.dir + (int64_t)i * F.d;
    double pen = 0.0;
    for (int k = threadIdx.x; k < F.d; k += blockDim.x) {
        const double x = th[k] + s * dr[k];
        const float v = (float)x;
        if (k == 0)
            b[i] = v;
        else
            W[(int64_t)i * F.n + (k - 1)] = v;
        if (F.alpha > 0.0 && k >= 1 && k - 1 != i) pen += sqrt(x * x + F.eps);
    }
    if (F.alpha > 0.0) {
        pen = block_sum(pen, shp);
        if (threadIdx.x == 0) F.pen[i] = pen;
    }
}
__global__ void fit_trial_kernel(FitState F, float* __restrict__ W, float* __restrict__ b) {
    fit_trial_body(F, blockIdx.x, W, b);
}

// Armijo test of every open line search against the rows' trial log-likelihoods
__device__ __forceinline__ void fit_armijo_body(const FitState& F, int32_t i, const double* __restrict__ Ltrial,
                                                double c1, int max_halvings) {
    if (i >= F.n || F.status[i] != ACTIVE || !F.pend[i]) return;
    const double Lt = Ltrial[i] - F.alpha * (F.alpha > 0.0 ? F.pen[i] : 0.0);  // penalised (Eq. 16)
    const double s = F.step[i], gd = F.gd[i];
    // f(trial) <= f + c1 s g.d   with f = -L
    if (isfinite(Lt) && -Lt <= -F.Lcur[i] + c1 * s * gd) {
        F.pend[i] = 0;
        F.acc[i] = 1;
        return;
    }
    // backtrack: minimiser of phi(0) = f, phi'(0) = g.d, phi(s) = f(trial), kept within [0.1 s, 0.5 s].
    // The Armijo failure gives f(trial) - f - s g.d > (1 - c1) s |g.d| > 0, so the quadratic is convex.
    double sn = 0.1 * s;
    if (isfinite(Lt)) {
        const double den = 2.0 * ((-Lt) - (-F.Lcur[i]) - gd * s);
        sn = fmin(fmax(-gd * s * s / den, 0.1 * s), 0.5 * s);
    }
    F.step[i] = sn;
    // below the floor the gain is smaller than the evaluation's own error
    const bool tiny = sn * fabs(gd) < F.floor * (fabs(F.Lcur[i]) + F.qd[i]);
    if (++F.halv[i] >= max_halvings || tiny) {
        F.pend[i] = 0;
        F.acc[i] = 0;
        if (F.hn[i] > 0) {
            // a poor quasi-Newton direction also shows a tiny predicted gain: retry from the gradient
            F.hn[i] = 0;
            F.hs[i] = 0;
        } else {
            F.status[i] = tiny ? GLM_ROW_AT_FLOOR : GLM_ROW_STALLED;
            atomicAdd(F.counters + 2, 1);
        }
        return;
    }
    atomicAdd(F.counters + 1, 1);
}
__global__ void fit_armijo_kernel(FitState F, const double* __restrict__ Ltrial, double c1, int max_halvings) {
    fit_armijo_body(F, blockIdx.x * blockDim.x + threadIdx.x, Ltrial, c1, max_halvings);
}

// accept the steps: theta += s d for accepted rows (block per row)
__device__ __forceinline__ void fit_commit_body(const FitState& F, int32_t i) {
    if (F.status[i] != ACTIVE || !F.acc[i]) return;
    const double s = F.step[i];
    double* th = F.theta + (int64_t)i * F.d;
    const double* dr = F.dir + (int64_t)i * F.d;
    for (int k = threadIdx.x; k < F.d; k += blockDim.x) th[k] += s * dr[k];
}
__global__ void fit_commit_kernel(FitState F) { fit_commit_body(F, blockIdx.x); }

// new gradient, curvature pair, stopping rule (block per row)
__device__ __forceinline__ void fit_update_body(const FitState& F, int32_t i, const double* __restrict__ Lnew,
                                                const double* __restrict__ G, const double* __restrict__ gb,
                                                double eta, int max_iter) {
    __shared__ double sh[32];
    if (F.status[i] != ACTIVE || !F.acc[i]) return;
    double* g = F.g + (int64_t)i * F.d;
    const double s = F.step[i];
    const double* dr = F.dir + (int64_t)i * F.d;
    const int slot = (F.hn[i] < F.m) ? (F.hs[i] + F.hn[i]) % F.m : F.hs[i];
    double* Sv = F.S + ((int64_t)slot * F.n + i) * F.d;
    double* Yv = F.Y + ((int64_t)slot * F.n + i) * F.d;
    double sy = 0.0;
    const double* th = F.theta + (int64_t)i * F.d;
    for (int k = threadIdx.x; k < F.d; k += blockDim.x) {
        const double gn = (k == 0) ? -gb[i] : -G[(int64_t)i * F.n + (k - 1)] + pen_grad(F, i, k, th[k]);
        const double y = gn - g[k];
        const double sv = s * dr[k];
        if (F.method == GLM_FIT_LBFGS) {
            Sv[k] = sv;
            Yv[k] = y;
        }
        sy += sv * y;
        g[k] = gn;
    }
    sy = block_sum(sy, sh);
    if (threadIdx.x == 0) {
        if (F.method == GLM_FIT_LBFGS && sy > 0.0) {
            F.rho[(int64_t)slot * F.n + i] = 1.0 / sy;
            if (F.hn[i] < F.m)
                F.hn[i]++;
            else
                F.hs[i] = (F.hs[i] + 1) % F.m;
        }
        const double Lold = F.Lcur[i], Ln = Lnew[i] - (F.alpha > 0.0 ? F.alpha * F.pen[i] : 0.0);
        F.Lcur[i] = Ln;
        F.gastep[i] = s;
        F.iters[i]++;
        if (fabs(Ln - Lold) < eta * fabs(Lold))
            F.status[i] = GLM_ROW_CONVERGED;
        else if (F.iters[i] >= max_iter)
            F.status[i] = GLM_ROW_MAXITER;
    }
}
__global__ void fit_update_kernel(FitState F, const double* __restrict__ Lnew, const double* __restrict__ G,
                                  const double* __restrict__ gb, double eta, int max_iter) {
    fit_update_body(F, blockIdx.x, Lnew, G, gb, eta, max_iter);
}

// gradient of -L at the start point
__global__ void fit_grad0_kernel(FitState F, const double* __restrict__ L, const double* __restrict__ G,
                                 const double* __restrict__ gb) {
    const int32_t i = blockIdx.x;
    double* g = F.g + (int64_t)i * F.d;
    const double* th = F.theta + (int64_t)i * F.d;
    for (int k = threadIdx.x; k < F.d; k += blockDim.x)
        g[k] = (k == 0) ? -gb[i] : -G[(int64_t)i * F.n + (k - 1)] + pen_grad(F, i, k, th[k]);
    if (threadIdx.x == 0) F.Lcur[i] = L[i] - (F.alpha > 0.0 ? F.alpha * F.pen[i] : 0.0);
}

// search direction and initial step of every active row (block per row)
__device__ __forceinline__ void fit_direction_body(const FitState& F, int32_t i) {
    __shared__ double sh[32];
    __shared__ double alpha[32];
    if (F.status[i] != ACTIVE) return;
    if (F.pend[i]) {  // a search still open (batched fits): it keeps its direction and step
        if (threadIdx.x == 0) atomicAdd(F.counters + 0, 1);
        return;
    }
    const double* g = F.g + (int64_t)i * F.d;
    double* q = F.dir + (int64_t)i * F.d;
    const int hn = (F.method == GLM_FIT_LBFGS) ? F.hn[i] : 0;
    const int hs = F.hs[i];
    for (int k = threadIdx.x; k < F.d; k += blockDim.x) q[k] = g[k];
    __syncthreads();
    if (hn > 0) {
        for (int h = hn - 1; h >= 0; --h) {
            const int sl = (hs + h) % F.m;
            const double* Sv = F.S + ((int64_t)sl * F.n + i) * F.d;
            const double* Yv = F.Y + ((int64_t)sl * F.n + i) * F.d;
            double p = 0.0;
            for (int k = threadIdx.x; k < F.d; k += blockDim.x) p += Sv[k] * q[k];
            const double a = F.rho[(int64_t)sl * F.n + i] * block_sum(p, sh);
            if (threadIdx.x == 0) alpha[h] = a;
            for (int k = threadIdx.x; k < F.d; k += blockDim.x) q[k] -= a * Yv[k];
            __syncthreads();
        }
        const int last = (hs + hn - 1) % F.m;
        const double* Sl = F.S + ((int64_t)last * F.n + i) * F.d;
        const double* Yl = F.Y + ((int64_t)last * F.n + i) * F.d;
        double sy = 0.0, yy = 0.0;
        for (int k = threadIdx.x; k < F.d; k += blockDim.x) {
            sy += Sl[k] * Yl[k];
            yy += Yl[k] * Yl[k];
        }
        sy = block_sum(sy, sh);
        yy = block_sum(yy, sh);
        const double gamma = sy / yy;
        for (int k = threadIdx.x; k < F.d; k += blockDim.x) q[k] *= gamma;
        __syncthreads();
        for (int h = 0; h < hn; ++h) {
            const int sl = (hs + h) % F.m;
            const double* Sv = F.S + ((int64_t)sl * F.n + i) * F.d;
            const double* Yv = F.Y + ((int64_t)sl * F.n + i) * F.d;
            double p = 0.0;
            for (int k = threadIdx.x; k < F.d; k += blockDim.x) p += Yv[k] * q[k];
            const double beta = F.rho[(int64_t)sl * F.n + i] * block_sum(p, sh);
            const double a = alpha[h];
            for (int k = threadIdx.x; k < F.d; k += blockDim.x) q[k] += (a - beta) * Sv[k];
            __syncthreads();
        }
    }
    // q now holds H g: the direction is -q
    double gq = 0.0, gg = 0.0;
    for (int k = threadIdx.x; k < F.d; k += blockDim.x) {
        q[k] = -q[k];
        gq += g[k] * q[k];
        gg += g[k] * g[k];
    }
    gq = block_sum(gq, sh);
    gg = block_sum(gg, sh);
    bool reset = !(gq < 0.0);
    if (reset) {  // not a descent direction: restart from the gradient
        for (int k = threadIdx.x; k < F.d; k += blockDim.x) q[k] = -g[k];
        gq = -gg;
    }
    if (threadIdx.x == 0) {
        if (reset) F.hn[i] = 0;
        const double gn = sqrt(gg);
        if (gg == 0.0) {
            F.status[i] = GLM_ROW_CONVERGED;
            return;
        }
        double s0;
        if (F.method == GLM_FIT_LBFGS)
            s0 = (reset || hn == 0) ? fmin(1.0, 1.0 / gn) : 1.0;
        else
            s0 = F.gastep[i] > 0.0 ? 2.0 * F.gastep[i] : fmin(1.0, 1.0 / gn);
        F.step[i] = s0;
        F.gd[i] = gq;
        F.halv[i] = 0;
        F.pend[i] = 1;
        F.acc[i] = 0;
        atomicAdd(F.counters + 0, 1);
    }
}

__global__ void fit_direction_kernel(FitState F) { fit_direction_body(F, blockIdx.x); }

// The rows with an open line search, in increasing order (one block; chunked block scan).
__device__ __forceinline__ void fit_compact_body(const FitState& F, int32_t* __restrict__ rows) {
    __shared__ int32_t sh[1024];
    const int32_t per = (F.n + blockDim.x - 1) / blockDim.x;
    const int32_t r0 = min((int32_t)threadIdx.x * per, F.n), r1 = min(r0 + per, F.n);
    int32_t cnt = 0;
    for (int32_t i = r0; i < r1; ++i) cnt += (F.status[i] == ACTIVE && F.pend[i]) ? 1 : 0;
    sh[threadIdx.x] = cnt;
    __syncthreads();
    for (int d = 1; d < (int)blockDim.x; d <<= 1) {  // inclusive Hillis-Steele scan
        const int32_t v = (threadIdx.x >= (unsigned)d) ? sh[threadIdx.x - d] : 0;
        __syncthreads();
        sh[threadIdx.x] += v;
        __syncthreads();
    }
    int32_t pos = sh[threadIdx.x] - cnt;
    for (int32_t i = r0; i < r1; ++i)
        if (F.status[i] == ACTIVE && F.pend[i]) rows[pos++] = i;
    if (threadIdx.x == blockDim.x - 1) F.counters[3] = sh[threadIdx.x];  // rows to evaluate
}
__global__ void fit_compact_kernel(FitState F, int32_t* __restrict__ rows) { fit_compact_body(F, rows); }

__global__ void fit_write_kernel(FitState F, float* __restrict__ W, float* __restrict__ b) {
    const int32_t i = blockIdx.x;
    const double* th = F.theta + (int64_t)i * F.d;
    for (int k = threadIdx.x; k < F.d; k += blockDim.x) {
        if (k == 0)
            b[i] = (float)th[0];
        else
            W[(int64_t)i * F.n + (k - 1)] = (float)th[k];
    }
}

__global__ void fit_finish_kernel(FitState F) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < F.n && F.status[i] == ACTIVE) F.status[i] = GLM_ROW_MAXITER;
}

}  // namespace

namespace {

// One problem's optimiser state: device pointers into its fit_mem.
struct FitProb {
    glm_ctx* c = nullptr;
    FitState F;
    double *G = nullptr, *gb = nullptr, *Lr = nullptr;
    int32_t* eval_rows = nullptr;  // rows of the current line-search round
    float *W32 = nullptr, *b32 = nullptr;
    float *W = nullptr, *b = nullptr;  // caller's output (and warm start)
    int iters = 0, evals = 0, grads = 0;
};

int fit_setup(glm_ctx* c, const glm_fit_opts_t* o, float* W, float* b, FitProb* fp) {
    const Problem& P = c->pb;
    Buffers& B = c->buf;
    const int32_t n = P.n, d = n + 1, m = o->m;
    // optimiser state: allocated once per problem (freed with the problem's workspace)
    if (!B.fit_mem || B.fit_m != m) {
        if (B.fit_mem) return set_error(c, GLM_ERR_UNSUPPORTED, "glm_fit: the L-BFGS memory cannot change within a problem");
        const size_t nd = (size_t)n * d;
        const size_t bytes = sizeof(double) * (nd * (3 + 2 * (size_t)m) + (size_t)m * n + 5 * (size_t)n + (size_t)n * n + n + n) +
                             sizeof(int32_t) * 8 * (size_t)n + sizeof(float) * ((size_t)n * n + n) + 64;
        int rc = ws_alloc_bytes(c, &B.fit_mem, bytes);
        if (rc) return rc;
        B.fit_m = m;
    }
    FitState& F = fp->F;
    F.n = n;
    F.d = d;
    F.m = m;
    F.method = o->method;
    F.qd = B.qd;
    // gains below this fraction of |L_i| + q_i are not resolved by the evaluation (the 16-bit forms carry
    // a gradient error of ~1e-4 of its terms, the plain FP32 form ~1e-9 of L)
    F.floor = o->gain_floor >= 0.0 ? o->gain_floor : (P.prec == GLM_PREC_F32) ? 1e-13 : 1e-10;
    F.alpha = o->alpha;
    F.eps = o->eps;
    const size_t nd = (size_t)n * d;
    double* dp = reinterpret_cast<double*>(B.fit_mem);
    F.theta = dp;
    dp += nd;
    F.g = dp;
    dp += nd;
    F.dir = dp;
    dp += nd;
    F.S = dp;
    dp += (size_t)m * nd;
    F.Y = dp;
    dp += (size_t)m * nd;
    F.rho = dp;
    dp += (size_t)m * n;
    F.Lcur = dp;
    dp += n;
    F.step = dp;
    dp += n;
    F.gd = dp;
    dp += n;
    F.gastep = dp;
    dp += n;
    F.pen = dp;
    dp += n;
    fp->G = dp;
    dp += (size_t)n * n;
    fp->gb = dp;
    dp += n;
    fp->Lr = dp;
    dp += n;
    int32_t* ip = reinterpret_cast<int32_t*>(dp);
    F.status = ip;
    ip += n;
    F.pend = ip;
    ip += n;
    F.acc = ip;
    ip += n;
    F.halv = ip;
    ip += n;
    F.hn = ip;
    ip += n;
    F.hs = ip;
    ip += n;
    F.iters = ip;
    ip += n;
    fp->eval_rows = ip;
    ip += n;
    float* flp = reinterpret_cast<float*>(ip);
    fp->W32 = flp;
    flp += (size_t)n * n;
    fp->b32 = flp;
    flp += n;
    F.counters = reinterpret_cast<int*>((reinterpret_cast<uintptr_t>(flp) + 15) & ~(uintptr_t)15);
    fp->c = c;
    fp->W = W;
    fp->b = b;
    return GLM_OK;
}

int ck(glm_ctx* c, cudaError_t e) { return e == cudaSuccess ? GLM_OK : set_error(c, GLM_ERR_CUDA, cudaGetErrorString(e)); }

// Start point, its log-likelihood and gradient.
int fit_start(FitProb& fp, const glm_fit_opts_t* o) {
    glm_ctx* c = fp.c;
    const Problem& P = c->pb;
    const int32_t n = P.n;
    cudaStream_t st = c->stream;
    int rc;
    fit_init_kernel<<<n, FT, 0, st>>>(fp.F, P.span, c->buf.qd, o->warm_start, fp.W, fp.b, c->row_r0,
                                      c->row_r1 < 0 ? n : c->row_r1);
    fit_trial_kernel<<<n, FT, 0, st>>>(fp.F, fp.W32, fp.b32);
    c->launches += 2;
    if ((rc = ck(c, reset_flags(c)))) return rc;
    if ((rc = eval_enqueue(c, fp.W32, fp.b32, fp.Lr, fp.G, fp.gb, true, false))) return rc;
    fp.evals++;
    fp.grads++;
    fit_grad0_kernel<<<n, FT, 0, st>>>(fp.F, fp.Lr, fp.G, fp.gb);
    c->launches += 1;
    return GLM_OK;
}

// Returned point, final log-likelihood, row states and report.
int fit_end(FitProb& fp, int8_t* row_status, glm_fit_report_t* rep, double seconds) {
    glm_ctx* c = fp.c;
    const int32_t n = c->pb.n;
    cudaStream_t st = c->stream;
    int rc;
    fit_finish_kernel<<<(n + 255) / 256, 256, 0, st>>>(fp.F);
    fit_write_kernel<<<n, FT, 0, st>>>(fp.F, fp.W, fp.b);
    fit_trial_kernel<<<n, FT, 0, st>>>(fp.F, fp.W32, fp.b32);
    c->launches += 3;
    if ((rc = eval_enqueue(c, fp.W32, fp.b32, fp.Lr, nullptr, nullptr, false, false))) return rc;
    fp.evals++;
    std::vector<int32_t> stat(n);
    std::vector<double> Lh(n);
    if ((rc = ck(c, cudaMemcpyAsync(stat.data(), fp.F.status, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st))))
        return rc;
    if ((rc = ck(c, cudaMemcpyAsync(Lh.data(), fp.Lr, sizeof(double) * n, cudaMemcpyDeviceToHost, st)))) return rc;
    if ((rc = eval_status(c))) return rc;
    int cnt[6] = {0, 0, 0, 0, 0, 0};
    double Ltot = 0.0;
    for (int32_t i = 0; i < n; ++i) {
        const int s = stat[i];
        if (s >= 0 && s < 6) cnt[s]++;
        if (row_status) row_status[i] = (int8_t)s;
        Ltot += Lh[i];
    }
    if (rep) {
        rep->iterations = fp.iters;
        rep->evaluations = fp.evals;
        rep->gradients = fp.grads;
        rep->converged = cnt[GLM_ROW_CONVERGED];
        rep->maxiter = cnt[GLM_ROW_MAXITER];
        rep->stalled = cnt[GLM_ROW_STALLED];
        rep->degenerate = cnt[GLM_ROW_DEGENERATE];
        rep->at_floor = cnt[GLM_ROW_AT_FLOOR];
        rep->excluded = cnt[GLM_ROW_EXCLUDED];
        rep->L = Ltot;
        rep->seconds = seconds;
    }
    if (cnt[GLM_ROW_MAXITER]) return GLM_STATUS_NOT_CONVERGED;
    if (cnt[GLM_ROW_STALLED]) return GLM_STATUS_STALLED;
    return GLM_OK;
}

}  // namespace

int fit_run(glm_ctx* c, const glm_fit_opts_t* o, float* W, float* b, int8_t* row_status, glm_fit_report_t* rep) {
    const auto t_start = std::chrono::steady_clock::now();
    const int32_t n = c->pb.n;
    FitProb fp;
    int rc;
    if ((rc = fit_setup(c, o, W, b, &fp))) return rc;
    FitState& F = fp.F;
    cudaStream_t st = c->stream;
    if ((rc = fit_start(fp, o))) return rc;
    int host_cnt[3] = {0, 0, 0};
    while (true) {
        if ((rc = ck(c, cudaMemsetAsync(F.counters, 0, 4 * sizeof(int), st)))) return rc;
        fit_direction_kernel<<<n, FT, 0, st>>>(F);
        c->launches += 1;
        if ((rc = ck(c, cudaMemcpyAsync(host_cnt, F.counters, 2 * sizeof(int), cudaMemcpyDeviceToHost, st)))) return rc;
        if ((rc = eval_status(c))) return rc;
        if (host_cnt[0] == 0 || fp.iters >= o->max_iter) break;
        // line search: every round evaluates the trial points of the rows whose search is still open, in
        // one batched product over just those rows; their rates and per-tile sums land at their own row
        // positions, so an accepted row keeps the values of its accepted point until the gradient.
        int32_t open = host_cnt[0];
        while (true) {
            fit_trial_kernel<<<n, FT, 0, st>>>(F, fp.W32, fp.b32);
            fit_compact_kernel<<<1, 1024, 0, st>>>(F, fp.eval_rows);
            c->launches += 2;
            if ((rc = eval_enqueue(c, fp.W32, fp.b32, fp.Lr, nullptr, nullptr, false, false, false, fp.eval_rows, open)))
                return rc;
            fp.evals++;
            if ((rc = ck(c, cudaMemsetAsync(F.counters + 1, 0, 2 * sizeof(int), st)))) return rc;
            fit_armijo_kernel<<<(n + 255) / 256, 256, 0, st>>>(F, fp.Lr, o->c1, o->max_halvings);
            c->launches += 1;
            if ((rc = ck(c, cudaMemcpyAsync(host_cnt + 1, F.counters + 1, 2 * sizeof(int), cudaMemcpyDeviceToHost, st))))
                return rc;
            // a non-finite trial only fails the Armijo test; clear the flag before it is read
            if ((rc = ck(c, cudaStreamSynchronize(st)))) return rc;
            if ((rc = ck(c, reset_flags(c)))) return rc;
            if (host_cnt[1] == 0) break;
            open = host_cnt[1];
        }
        // accepted points: gradient there, from the rates and per-tile sums each accepted row left in
        // its acceptance round.  Rows not accepted (stopped, restarting) take nothing from it.
        fit_commit_kernel<<<n, FT, 0, st>>>(F);
        c->launches += 1;
        if ((rc = eval_enqueue(c, fp.W32, fp.b32, fp.Lr, fp.G, fp.gb, true, true))) return rc;
        fp.grads++;
        fit_update_kernel<<<n, FT, 0, st>>>(F, fp.Lr, fp.G, fp.gb, o->eta, o->max_iter);
        c->launches += 1;
        fp.iters++;
    }
    return fit_end(fp, row_status, rep,
                   std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count());
}

// ---- several problems at once ----
//
// Every problem keeps its own optimiser state; the two contractions of each evaluation are one launch
// over all problems (tensor-core forms).  One iteration - directions, GRAPH_ROUNDS line-search rounds,
// gradient, update - is recorded once as a CUDA graph and replayed; the host reads one count per
// problem after each replay.  A row whose search is still open after the rounds of an iteration keeps
// its direction and step and goes on searching in the next one.

namespace {

constexpr int GRAPH_ROUNDS = 3;
constexpr int FB_MAX = 32;

// Every problem of a batched fit, for kernels that run over the rows of all problems at once (device
// memory).  Global row r belongs to problem p with rbeg[p] <= r < rbeg[p + 1].
struct FitBatch {
    int32_t np;
    int32_t rbeg[FB_MAX + 1];  // rows
    int64_t ebeg[FB_MAX + 1];  // n x n elements
    int64_t wbeg[FB_MAX + 1];  // W-split elements (n x ldk)
    FitState F[FB_MAX];
    float* W32[FB_MAX];
    float* b32[FB_MAX];
    double* Lr[FB_MAX];
    double* G[FB_MAX];
    double* gb[FB_MAX];
    int32_t* rows[FB_MAX];
    const double* part_e[FB_MAX];
    const double* part_s[FB_MAX];
    const double* qd[FB_MAX];
    const double* C[FB_MAX];
    const float* part_g[FB_MAX];
    int64_t ntile[FB_MAX];
    int32_t planes[FB_MAX];  // planes of part_e / part_s (1: the grid form, the only one batched)
    int32_t nsplit[FB_MAX];
    double dt[FB_MAX];
    int* flags[FB_MAX];
    double* eb[FB_MAX];
    void* Wsplit[FB_MAX];
    int64_t ldk[FB_MAX];
};

__device__ __forceinline__ int fb_prob(const int32_t* beg, int np, int64_t r) {
    int p = 0;
    while (p + 1 < np && r >= beg[p + 1]) ++p;
    return p;
}
__device__ __forceinline__ int fb_prob64(const int64_t* beg, int np, int64_t r) {
    int p = 0;
    while (p + 1 < np && r >= beg[p + 1]) ++p;
    return p;
}

// iteration start: counters of every problem
__global__ void fb_start_kernel(const FitBatch* __restrict__ B) {
    const int p = threadIdx.x;
    if (p < B->np) {
        int* c = B->F[p].counters;
        c[0] = c[1] = c[2] = 0;
    }
}
// after a round: the open-search counts and the error flags (a non-finite trial only fails its Armijo test)
__global__ void fb_round_reset_kernel(const FitBatch* __restrict__ B) {
    const int p = threadIdx.x;
    if (p < B->np) {
        B->F[p].counters[1] = B->F[p].counters[2] = 0;
        B->flags[p][0] = B->flags[p][1] = 0;
    }
}
__global__ void fb_direction_kernel(const FitBatch* __restrict__ B) {
    const int p = fb_prob(B->rbeg, B->np, blockIdx.x);
    fit_direction_body(B->F[p], blockIdx.x - B->rbeg[p]);
}
__global__ void fb_trial_kernel(const FitBatch* __restrict__ B) {
    const int p = fb_prob(B->rbeg, B->np, blockIdx.x);
    fit_trial_body(B->F[p], blockIdx.x - B->rbeg[p], B->W32[p], B->b32[p]);
}
__global__ void fb_compact_kernel(const FitBatch* __restrict__ B) {
    fit_compact_body(B->F[blockIdx.x], B->rows[blockIdx.x]);
}
__global__ void fb_commit_kernel(const FitBatch* __restrict__ B) {
    const int p = fb_prob(B->rbeg, B->np, blockIdx.x);
    fit_commit_body(B->F[p], blockIdx.x - B->rbeg[p]);
}
__global__ void fb_armijo_kernel(const FitBatch* __restrict__ B, int32_t nrows, double c1, int max_halvings) {
    const int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    const int p = fb_prob(B->rbeg, B->np, r);
    fit_armijo_body(B->F[p], r - B->rbeg[p], B->Lr[p], c1, max_halvings);
}
__global__ void fb_update_kernel(const FitBatch* __restrict__ B, double eta, int max_iter) {
    const int p = fb_prob(B->rbeg, B->np, blockIdx.x);
    fit_update_body(B->F[p], blockIdx.x - B->rbeg[p], B->Lr[p], B->G[p], B->gb[p], eta, max_iter);
}
// exp(c), c = max(b_i, floor), of every row of every problem (the U product's e^U = e^c e^(U - c))
__global__ void fb_exp_bias_kernel(const FitBatch* __restrict__ B, int32_t nrows) {
    const int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    const int p = fb_prob(B->rbeg, B->np, r);
    const int32_t i = r - B->rbeg[p];
    const float bi = B->b32[p][i];
    const double v = exp((double)fmaxf(bi, EXP_SPLIT_FLOOR));
    if (!isfinite(bi) || !(v <= 1e300)) atomicOr(B->flags[p], 1);
    B->eb[p][i] = v;
}
// hi + lo parts of the rows to evaluate (rows[p][l], l < counters[3]) of every problem, packed per problem
template <typename T16>
__global__ void fb_split_w_kernel(const FitBatch* __restrict__ B, int64_t total) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const int p = fb_prob64(B->wbeg, B->np, e);
    const FitState& F = B->F[p];
    const int64_t ldk = B->ldk[p], el = e - B->wbeg[p];
    const int64_t l = el / ldk, k = el % ldk;
    if (l >= F.counters[3]) return;
    const int32_t i = B->rows[p][l];
    float w = (k < F.n) ? B->W32[p][(int64_t)i * F.n + k] : 0.f;
    if (!isfinite(w)) atomicOr(B->flags[p], 1);
    T16* hi = static_cast<T16*>(B->Wsplit[p]);
    T16* lo = hi + (int64_t)F.n * ldk;
    T16 h, lw;
    if constexpr (std::is_same<T16, __nv_bfloat16>::value) {
        h = __float2bfloat16_rn(w);
        lw = __float2bfloat16_rn(w - __bfloat162float(h));
    } else {
        h = __float2half_rn(w);
        lw = __float2half_rn(w - __half2float(h));
    }
    hi[el] = h;
    lo[el] = lw;
}
// L_i (and with gb the bias gradient) of every row of every problem from the per-tile partials (warp per row)
__global__ void fb_reduce_rows_kernel(const FitBatch* __restrict__ B, int32_t nrows, bool with_gb) {
    const int32_t r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= nrows) return;
    const int p = fb_prob(B->rbeg, B->np, r);
    const int32_t i = r - B->rbeg[p];
    const int64_t nt = B->ntile[p];
    const int64_t plane = (int64_t)(B->rbeg[p + 1] - B->rbeg[p]) * nt;
    double integ = 0.0, spk = 0.0;
    for (int pl = 0; pl < B->planes[p]; ++pl) {
        const double* pe = B->part_e[p] + pl * plane + (int64_t)i * nt;
        const double* ps = B->part_s[p] + pl * plane + (int64_t)i * nt;
        for (int64_t t = lane; t < nt; t += 32) {
            integ += pe[t];
            spk += ps[t];
        }
    }
    for (int off = 16; off >= 1; off >>= 1) {
        integ += __shfl_xor_sync(0xffffffffu, integ, off);
        spk += __shfl_xor_sync(0xffffffffu, spk, off);
    }
    if (lane == 0) {
        const double q = B->qd[p][i];
        B->Lr[p][i] = q * (double)B->b32[p][i] + spk - B->dt[p] * integ;
        if (with_gb) B->gb[p][i] = q - B->dt[p] * integ;
    }
}
// G = C - sum over splits of E X^T, every element of every problem
__global__ void fb_reduce_grad_kernel(const FitBatch* __restrict__ B, int64_t total) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const int p = fb_prob64(B->ebeg, B->np, e);
    const int64_t el = e - B->ebeg[p], nn = B->ebeg[p + 1] - B->ebeg[p];
    // FP32 pair summed with TwoSum, one FP64 value at the end (as reduce_grad_kernel: FP64 adds are scarce)
    float hi = 0.f, lo = 0.f;
    for (int k = 0; k < B->nsplit[p]; ++k) {
        const float v = B->part_g[p][k * nn + el];
        const float s = hi + v, bp = s - hi;
        lo += (hi - (s - bp)) + (v - bp);
        hi = s;
    }
    B->G[p][el] = B->C[p][el] - ((double)hi + (double)lo);
}

// rows still active in each problem (block per problem)
__global__ void count_active_kernel(const int32_t* const* __restrict__ status, const int32_t* __restrict__ nrows,
                                    int* __restrict__ dst) {
    __shared__ int sh[32];
    const int p = blockIdx.x;
    const int32_t* st = status[p];
    int c = 0;
    for (int32_t i = threadIdx.x; i < nrows[p]; i += blockDim.x) c += st[i] == ACTIVE ? 1 : 0;
    for (int off = 16; off >= 1; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        dst[p] = t;
    }
}

}  // namespace

int fit_run_batch(glm_ctx* const* cs, int np, const glm_fit_opts_t* o, float* const* W, float* const* b,
                  int8_t* const* row_status, glm_fit_report_t* reps) {
    const auto t_start = std::chrono::steady_clock::now();
    glm_ctx* c0 = cs[0];
    // the batch runs on a private stream (a CUDA graph cannot be recorded on the legacy default stream),
    // ordered after the work already queued on the first context's stream
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
        return set_error(c0, GLM_ERR_CUDA, "cudaStreamCreateWithFlags");
    {
        cudaEvent_t ev;
        cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(ev, c0->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev, 0);
        cudaEventDestroy(ev);
        if (e != cudaSuccess) {
            cudaStreamDestroy(st);
            return set_error(c0, GLM_ERR_CUDA, cudaGetErrorString(e));
        }
    }
    std::vector<cudaStream_t> saved(np);
    std::vector<bool> saved_prof(np);
    for (int p = 0; p < np; ++p) {  // all work of the batch goes to the first context's stream
        saved[p] = cs[p]->stream;
        saved_prof[p] = cs[p]->prof_on;
        cs[p]->stream = st;
    }
    std::vector<FitProb> fp(np);
    void *host_u = nullptr, *host_g = nullptr, *dev_u = nullptr, *dev_g = nullptr, *dev_aux = nullptr, *fb_mem = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int rc = GLM_OK;
    auto done = [&](int r) {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        cudaFree(dev_u);
        cudaFree(dev_g);
        cudaFree(dev_aux);
        cudaFree(fb_mem);
        std::free(host_u);
        std::free(host_g);
        cudaStreamSynchronize(st);
        for (int p = 0; p < np; ++p) {
            cs[p]->stream = saved[p];
            cs[p]->prof_on = saved_prof[p];
        }
        cudaStreamDestroy(st);
        return r;
    };
    for (int p = 0; p < np && !rc; ++p) rc = fit_setup(cs[p], o, W[p], b[p], &fp[p]);
    if (rc) return done(rc);
    // batch descriptors, the per-problem count pointers and the gathered counts
    std::vector<float*> W32(np), b32(np);
    std::vector<int32_t*> rows(np);
    std::vector<const int32_t*> mdev(np);
    std::vector<const int32_t*> st_src(np);
    std::vector<int32_t> nrows(np);
    for (int p = 0; p < np; ++p) {
        W32[p] = fp[p].W32;
        b32[p] = fp[p].b32;
        rows[p] = fp[p].eval_rows;
        mdev[p] = fp[p].F.counters + 3;  // set by fit_compact_kernel
        st_src[p] = fp[p].F.status;
        nrows[p] = fp[p].F.n;
    }
    const size_t bb = tc_batch_bytes();
    host_u = std::malloc(bb);
    host_g = std::malloc(bb);
    if (!host_u || !host_g) return done(set_error(c0, GLM_ERR_OOM, "host memory"));
    if ((rc = tc_batch_fill(cs, np, W32.data(), b32.data(), rows.data(), mdev.data(), host_u, host_g)))
        return done(set_error(c0, rc, "bad batch"));
    const size_t aux = sizeof(int32_t*) * np + 2 * sizeof(int) * np;
    if ((rc = ck(c0, cudaMalloc(&dev_u, bb))) || (rc = ck(c0, cudaMalloc(&dev_g, bb))) ||
        (rc = ck(c0, cudaMalloc(&dev_aux, aux))))
        return done(rc);
    const int32_t** d_src = static_cast<const int32_t**>(dev_aux);
    int32_t* d_n = reinterpret_cast<int32_t*>(d_src + np);
    int* d_cnt = d_n + np;
    if ((rc = ck(c0, cudaMemcpy(dev_u, host_u, bb, cudaMemcpyHostToDevice))) ||
        (rc = ck(c0, cudaMemcpy(dev_g, host_g, bb, cudaMemcpyHostToDevice))) ||
        (rc = ck(c0, cudaMemcpy(d_src, st_src.data(), sizeof(int32_t*) * np, cudaMemcpyHostToDevice))) ||
        (rc = ck(c0, cudaMemcpy(d_n, nrows.data(), sizeof(int32_t) * np, cudaMemcpyHostToDevice))))
        return done(rc);
    // the batched E X^T launch is tuned as a whole (row tile and splits), then skips finished problems
    if ((rc = tc_autotune_batch(cs, np, dev_g, host_g))) return done(set_error(c0, rc, "batch autotune failed"));
    {
        std::vector<const int*> cnt_ptr(np);
        for (int p = 0; p < np; ++p) cnt_ptr[p] = d_cnt + p;
        tc_batch_set_grad_counts(host_g, np, cnt_ptr.data());
        std::vector<int> init(np);
        for (int p = 0; p < np; ++p) init[p] = fp[p].F.n;
        if ((rc = ck(c0, cudaMemcpy(d_cnt, init.data(), sizeof(int) * np, cudaMemcpyHostToDevice))) ||
            (rc = ck(c0, cudaMemcpy(dev_g, host_g, tc_batch_bytes(), cudaMemcpyHostToDevice))))
            return done(rc);
    }
    for (int p = 0; p < np && !rc; ++p) rc = fit_start(fp[p], o);
    if (rc) return done(rc);
    if ((rc = ck(c0, cudaStreamSynchronize(st)))) return done(rc);
    for (int p = 0; p < np && !rc; ++p) rc = eval_status(cs[p]);
    if (rc) return done(rc);

    // the batch-wide view of every problem, for the kernels that run over all rows at once
    FitBatch hb;
    std::memset(static_cast<void*>(&hb), 0, sizeof(hb));
    hb.np = np;
    for (int p = 0; p < np; ++p) {
        glm_ctx* c = cs[p];
        const int64_t n = c->pb.n;
        hb.rbeg[p + 1] = hb.rbeg[p] + (int32_t)n;
        hb.ebeg[p + 1] = hb.ebeg[p] + n * n;
        hb.wbeg[p + 1] = hb.wbeg[p] + n * c->buf.ldn;
        hb.F[p] = fp[p].F;
        hb.W32[p] = fp[p].W32;
        hb.b32[p] = fp[p].b32;
        hb.Lr[p] = fp[p].Lr;
        hb.G[p] = fp[p].G;
        hb.gb[p] = fp[p].gb;
        hb.rows[p] = fp[p].eval_rows;
        hb.part_e[p] = c->buf.part_e;
        hb.part_s[p] = c->buf.part_s;
        hb.qd[p] = c->buf.qd;
        hb.C[p] = c->buf.C;
        hb.part_g[p] = c->buf.part_g;
        hb.ntile[p] = c->pb.Tpad / tc_tile_t();
        hb.planes[p] = c->pb.ct ? CT_PARTS : 1;
        hb.nsplit[p] = tc_nsplit(c);
        hb.dt[p] = c->pb.dt_int;
        hb.flags[p] = c->buf.flags;
        hb.eb[p] = c->buf.eb;
        hb.Wsplit[p] = c->buf.Wsplit;
        hb.ldk[p] = c->buf.ldn;
    }
    FitBatch* d_fb = nullptr;
    if ((rc = ck(c0, cudaMalloc(&d_fb, sizeof(FitBatch))))) return done(rc);
    fb_mem = d_fb;
    if ((rc = ck(c0, cudaMemcpy(d_fb, &hb, sizeof(FitBatch), cudaMemcpyHostToDevice)))) return done(rc);
    const int32_t rows_all = hb.rbeg[np];
    const int64_t nelem = hb.ebeg[np], nw = hb.wbeg[np];
    const bool bf = c0->pb.prec == GLM_PREC_BF16;

    // one iteration, recorded once: every kernel runs over all problems
    int64_t launches = 0;
    auto enqueue_iteration = [&]() -> int {
        int r;
        fb_start_kernel<<<1, FB_MAX, 0, st>>>(d_fb);
        fb_direction_kernel<<<rows_all, FT, 0, st>>>(d_fb);
        launches += 2;
        for (int round = 0; round < GRAPH_ROUNDS; ++round) {
            fb_trial_kernel<<<rows_all, FT, 0, st>>>(d_fb);
            fb_compact_kernel<<<np, 1024, 0, st>>>(d_fb);
            fb_exp_bias_kernel<<<(rows_all + 255) / 256, 256, 0, st>>>(d_fb, rows_all);
            if (bf)
                fb_split_w_kernel<__nv_bfloat16><<<(unsigned)((nw + 255) / 256), 256, 0, st>>>(d_fb, nw);
            else
                fb_split_w_kernel<__half><<<(unsigned)((nw + 255) / 256), 256, 0, st>>>(d_fb, nw);
            if ((r = ck(c0, launch_tc_u_batch(c0, dev_u)))) return r;
            fb_reduce_rows_kernel<<<(rows_all + 7) / 8, 256, 0, st>>>(d_fb, rows_all, false);
            fb_armijo_kernel<<<(rows_all + 255) / 256, 256, 0, st>>>(d_fb, rows_all, o->c1, o->max_halvings);
            fb_round_reset_kernel<<<1, FB_MAX, 0, st>>>(d_fb);
            launches += 8;
            for (int p = 0; p < np; ++p) fp[p].evals++;
        }
        fb_commit_kernel<<<rows_all, FT, 0, st>>>(d_fb);
        if ((r = ck(c0, launch_tc_grad_batch(c0, dev_g)))) return r;
        fb_reduce_rows_kernel<<<(rows_all + 7) / 8, 256, 0, st>>>(d_fb, rows_all, true);
        fb_reduce_grad_kernel<<<(unsigned)((nelem + 255) / 256), 256, 0, st>>>(d_fb, nelem);
        fb_update_kernel<<<rows_all, FT, 0, st>>>(d_fb, o->eta, o->max_iter);
        count_active_kernel<<<np, 256, 0, st>>>(d_src, d_n, d_cnt);
        launches += 6;
        for (int p = 0; p < np; ++p) {
            fp[p].grads++;
            fp[p].iters++;
        }
        return GLM_OK;
    };
    for (int p = 0; p < np; ++p) cs[p]->prof_on = false;  // no event records inside the graph
    // attributes and a first pass outside capture
    if ((rc = enqueue_iteration())) return done(rc);
    const int64_t per_iteration = launches;
    std::vector<int> host_cnt(np, 0);
    auto read_counts = [&]() -> int {
        int r;
        if ((r = ck(c0, cudaMemcpyAsync(host_cnt.data(), d_cnt, sizeof(int) * np, cudaMemcpyDeviceToHost, st))))
            return r;
        if ((r = ck(c0, cudaStreamSynchronize(st)))) return r;
        for (int p = 0; p < np; ++p)
            if ((r = eval_status(cs[p]))) return r;
        return GLM_OK;
    };
    if ((rc = read_counts())) return done(rc);
    if ((rc = ck(c0, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal)))) return done(rc);
    const int cap_rc = enqueue_iteration();
    cudaError_t ce = cudaStreamEndCapture(st, &graph);
    if (cap_rc) return done(cap_rc);
    if ((rc = ck(c0, ce)) || (rc = ck(c0, cudaGraphInstantiate(&exec, graph, 0)))) return done(rc);
    // the recorded iteration also counted itself once: undo that
    for (int p = 0; p < np; ++p) {
        fp[p].iters--;
        fp[p].grads--;
        fp[p].evals -= GRAPH_ROUNDS;
    }
    int iter = 1;
    const int max_iter = o->max_iter + o->max_halvings;  // searches may run across iterations
    while (iter < max_iter) {
        bool any = false;
        for (int p = 0; p < np; ++p) any |= host_cnt[p] > 0;
        if (!any) break;
        if ((rc = ck(c0, cudaGraphLaunch(exec, st)))) return done(rc);
        for (int p = 0; p < np; ++p) {
            fp[p].iters++;
            fp[p].grads++;
            fp[p].evals += GRAPH_ROUNDS;
        }
        c0->launches += per_iteration;
        ++iter;
        if ((rc = read_counts())) return done(rc);
    }
    for (int p = 0; p < np; ++p) cs[p]->prof_on = saved_prof[p];
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    int worst = GLM_OK;
    for (int p = 0; p < np; ++p) {
        const int r = fit_end(fp[p], row_status ? row_status[p] : nullptr, reps ? &reps[p] : nullptr, secs);
        if (r < 0) return done(r);
        if (r > worst) worst = r;
    }
    return done(worst);
}

}  // namespace glm
