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

#include <chrono>
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
    int* counters;   // [3]  active rows, open line searches, rows stopped in this round
    const double* qd; // [n]  spike counts
    double floor;     // smallest predicted gain s |g.d| worth testing, relative to |L_i| + q_i
};

__global__ void fit_init_kernel(FitState F, int64_t T, double dt, const double* __restrict__ qd, int warm,
                                const float* __restrict__ W, const float* __restrict__ b) {
    const int32_t i = blockIdx.x;
    double* th = F.theta + (int64_t)i * F.d;
    const double q = qd[i];
    const bool degen = q == 0.0;
    for (int k = threadIdx.x; k < F.d; k += blockDim.x) {
        double v;
        if (k == 0)
            v = degen ? log(1e-3) : (warm ? (double)b[i] : log(q / ((double)T * dt)));
        else
            v = (degen || !warm) ? 0.0 : (double)W[(int64_t)i * F.n + (k - 1)];
        th[k] = v;
    }
    if (threadIdx.x == 0) {
        F.status[i] = degen ? GLM_ROW_DEGENERATE : ACTIVE;
        F.hn[i] = 0;
        F.hs[i] = 0;
        F.iters[i] = 0;
        F.pend[i] = 0;
        F.acc[i] = 0;
        F.gastep[i] = 0.0;
    }
}

// trial point in FP32 for the evaluator: theta + s d for rows with an open or accepted step, theta otherwise
__global__ void fit_trial_kernel(FitState F, float* __restrict__ W, float* __restrict__ b) {
    const int32_t i = blockIdx.x;
    const bool move = F.status[i] == ACTIVE && (F.pend[i] || F.acc[i]);
    const double s = move ? F.step[i] : 0.0;
    const double* th = F.theta + (int64_t)i * F.d;
    const double* dr = F.dir + (int64_t)i * F.d;
    for (int k = threadIdx.x; k < F.d; k += blockDim.x) {
        const float v = (float)(th[k] + s * dr[k]);
        if (k == 0)
            b[i] = v;
        else
            W[(int64_t)i * F.n + (k - 1)] = v;
    }
}

// Armijo test of every open line search against the rows' trial log-likelihoods
__global__ void fit_armijo_kernel(FitState F, const double* __restrict__ Ltrial, double c1, int max_halvings) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= F.n || F.status[i] != ACTIVE || !F.pend[i]) return;
    const double Lt = Ltrial[i];
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

// accept the steps: theta += s d for accepted rows (block per row)
__global__ void fit_commit_kernel(FitState F) {
    const int32_t i = blockIdx.x;
    if (F.status[i] != ACTIVE || !F.acc[i]) return;
    const double s = F.step[i];
    double* th = F.theta + (int64_t)i * F.d;
    const double* dr = F.dir + (int64_t)i * F.d;
    for (int k = threadIdx.x; k < F.d; k += blockDim.x) th[k] += s * dr[k];
}

// new gradient, curvature pair, stopping rule (block per row)
__global__ void fit_update_kernel(FitState F, const double* __restrict__ Lnew, const double* __restrict__ G,
                                  const double* __restrict__ gb, double eta, int max_iter) {
    __shared__ double sh[32];
    const int32_t i = blockIdx.x;
    if (F.status[i] != ACTIVE || !F.acc[i]) return;
    double* g = F.g + (int64_t)i * F.d;
    const double s = F.step[i];
    const double* dr = F.dir + (int64_t)i * F.d;
    const int slot = (F.hn[i] < F.m) ? (F.hs[i] + F.hn[i]) % F.m : F.hs[i];
    double* Sv = F.S + ((int64_t)slot * F.n + i) * F.d;
    double* Yv = F.Y + ((int64_t)slot * F.n + i) * F.d;
    double sy = 0.0;
    for (int k = threadIdx.x; k < F.d; k += blockDim.x) {
        const double gn = (k == 0) ? -gb[i] : -G[(int64_t)i * F.n + (k - 1)];
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
        const double Lold = F.Lcur[i], Ln = Lnew[i];
        F.Lcur[i] = Ln;
        F.gastep[i] = s;
        F.iters[i]++;
        if (fabs(Ln - Lold) < eta * fabs(Lold))
            F.status[i] = GLM_ROW_CONVERGED;
        else if (F.iters[i] >= max_iter)
            F.status[i] = GLM_ROW_MAXITER;
    }
}

// gradient of -L at the start point
__global__ void fit_grad0_kernel(FitState F, const double* __restrict__ L, const double* __restrict__ G,
                                 const double* __restrict__ gb) {
    const int32_t i = blockIdx.x;
    double* g = F.g + (int64_t)i * F.d;
    for (int k = threadIdx.x; k < F.d; k += blockDim.x) g[k] = (k == 0) ? -gb[i] : -G[(int64_t)i * F.n + (k - 1)];
    if (threadIdx.x == 0) F.Lcur[i] = L[i];
}

// search direction and initial step of every active row (block per row)
__global__ void fit_direction_kernel(FitState F) {
    __shared__ double sh[32];
    __shared__ double alpha[32];
    const int32_t i = blockIdx.x;
    if (F.status[i] != ACTIVE) return;
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

int fit_run(glm_ctx* c, const glm_fit_opts_t* o, float* W, float* b, int8_t* row_status, glm_fit_report_t* rep) {
    const auto t_start = std::chrono::steady_clock::now();
    const Problem& P = c->pb;
    Buffers& B = c->buf;
    const int32_t n = P.n, d = n + 1, m = o->m;
    // optimiser state: allocated once per problem (freed with the problem's workspace)
    if (!B.fit_mem || B.fit_m != m) {
        if (B.fit_mem) return set_error(c, GLM_ERR_UNSUPPORTED, "glm_fit: the L-BFGS memory cannot change within a problem");
        const size_t nd = (size_t)n * d;
        const size_t bytes = sizeof(double) * (nd * (3 + 2 * (size_t)m) + (size_t)m * n + 4 * (size_t)n + (size_t)n * n + n + n) +
                             sizeof(int32_t) * 7 * (size_t)n + sizeof(float) * ((size_t)n * n + n) + 64;
        int rc = ws_alloc_bytes(c, &B.fit_mem, bytes);
        if (rc) return rc;
        B.fit_m = m;
    }
    FitState F;
    F.n = n;
    F.d = d;
    F.m = m;
    F.method = o->method;
    F.qd = B.qd;
    // gains below this fraction of |L_i| + q_i are not resolved by the evaluation (the 16-bit forms carry
    // a gradient error of ~1e-4 of its terms, the plain FP32 form ~1e-9 of L)
    F.floor = o->gain_floor >= 0.0 ? o->gain_floor : (P.prec == GLM_PREC_F32) ? 1e-13 : 1e-10;
    {
        uint8_t* p = reinterpret_cast<uint8_t*>(B.fit_mem);
        const size_t nd = (size_t)n * d;
        double* dp = reinterpret_cast<double*>(p);
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
        double* G = dp;
        dp += (size_t)n * n;
        double* gb = dp;
        dp += n;
        double* Lr = dp;
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
        float* fp = reinterpret_cast<float*>(ip);
        float* W32 = fp;
        fp += (size_t)n * n;
        float* b32 = fp;
        fp += n;
        F.counters = reinterpret_cast<int*>((reinterpret_cast<uintptr_t>(fp) + 15) & ~(uintptr_t)15);

        cudaStream_t st = c->stream;
        int evals = 0, grads = 0, iters = 0;
        auto ck = [&](cudaError_t e) { return e == cudaSuccess ? GLM_OK : set_error(c, GLM_ERR_CUDA, cudaGetErrorString(e)); };
        int rc;
        fit_init_kernel<<<n, FT, 0, st>>>(F, P.T, P.dt, B.qd, o->warm_start, W, b);
        fit_trial_kernel<<<n, FT, 0, st>>>(F, W32, b32);
        c->launches += 2;
        if ((rc = ck(reset_flags(c)))) return rc;
        if ((rc = eval_enqueue(c, W32, b32, Lr, G, gb, true, false))) return rc;
        evals++;
        grads++;
        fit_grad0_kernel<<<n, FT, 0, st>>>(F, Lr, G, gb);
        c->launches += 1;
        int host_cnt[3] = {0, 0, 0};
        while (true) {
            if ((rc = ck(cudaMemsetAsync(F.counters, 0, 3 * sizeof(int), st)))) return rc;
            fit_direction_kernel<<<n, FT, 0, st>>>(F);
            c->launches += 1;
            if ((rc = ck(cudaMemcpyAsync(host_cnt, F.counters, 2 * sizeof(int), cudaMemcpyDeviceToHost, st)))) return rc;
            if ((rc = eval_status(c))) return rc;
            if (host_cnt[0] == 0 || iters >= o->max_iter) break;
            // line search: every round evaluates all rows' trial points in one batched product
            int rounds = 0;
            while (true) {
                fit_trial_kernel<<<n, FT, 0, st>>>(F, W32, b32);
                c->launches += 1;
                if ((rc = eval_enqueue(c, W32, b32, Lr, nullptr, nullptr, false, false))) return rc;
                evals++;
                if ((rc = ck(cudaMemsetAsync(F.counters + 1, 0, 2 * sizeof(int), st)))) return rc;
                fit_armijo_kernel<<<(n + 255) / 256, 256, 0, st>>>(F, Lr, o->c1, o->max_halvings);
                c->launches += 1;
                rounds++;
                if ((rc = ck(cudaMemcpyAsync(host_cnt + 1, F.counters + 1, 2 * sizeof(int), cudaMemcpyDeviceToHost, st))))
                    return rc;
                // a non-finite trial only fails the Armijo test; clear the flag before it is read
                if ((rc = ck(cudaStreamSynchronize(st)))) return rc;
                if ((rc = ck(reset_flags(c)))) return rc;
                if (host_cnt[1] == 0) break;
            }
            // accepted points: gradient there.  Every accepted row was evaluated at its accepted point in
            // each round since its acceptance, the last one included, so that round's U product and
            // per-tile sums serve the gradient.  Rows not accepted (stalled, restarting) take nothing
            // from this evaluation.
            fit_commit_kernel<<<n, FT, 0, st>>>(F);
            c->launches += 1;
            if ((rc = eval_enqueue(c, W32, b32, Lr, G, gb, true, true))) return rc;
            grads++;
            (void)rounds;
            fit_update_kernel<<<n, FT, 0, st>>>(F, Lr, G, gb, o->eta, o->max_iter);
            c->launches += 1;
            iters++;
        }
        fit_finish_kernel<<<(n + 255) / 256, 256, 0, st>>>(F);
        fit_write_kernel<<<n, FT, 0, st>>>(F, W, b);
        c->launches += 2;
        // final log-likelihood at the returned point
        fit_trial_kernel<<<n, FT, 0, st>>>(F, W32, b32);
        c->launches += 1;
        if ((rc = eval_enqueue(c, W32, b32, Lr, nullptr, nullptr, false, false))) return rc;
        evals++;
        std::vector<int32_t> stat(n);
        std::vector<double> Lh(n);
        if ((rc = ck(cudaMemcpyAsync(stat.data(), F.status, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st)))) return rc;
        if ((rc = ck(cudaMemcpyAsync(Lh.data(), Lr, sizeof(double) * n, cudaMemcpyDeviceToHost, st)))) return rc;
        if ((rc = eval_status(c))) return rc;
        int cnt[5] = {0, 0, 0, 0, 0};
        double Ltot = 0.0;
        for (int32_t i = 0; i < n; ++i) {
            const int s = stat[i];
            if (s >= 0 && s < 5) cnt[s]++;
            if (row_status) row_status[i] = (int8_t)s;
            Ltot += Lh[i];
        }
        if (rep) {
            rep->iterations = iters;
            rep->evaluations = evals;
            rep->gradients = grads;
            rep->converged = cnt[GLM_ROW_CONVERGED];
            rep->maxiter = cnt[GLM_ROW_MAXITER];
            rep->stalled = cnt[GLM_ROW_STALLED];
            rep->degenerate = cnt[GLM_ROW_DEGENERATE];
            rep->at_floor = cnt[GLM_ROW_AT_FLOOR];
            rep->L = Ltot;
            rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
        }
        if (cnt[GLM_ROW_MAXITER]) return GLM_STATUS_NOT_CONVERGED;
        if (cnt[GLM_ROW_STALLED]) return GLM_STATUS_STALLED;
        return GLM_OK;
    }
}

}  // namespace glm
