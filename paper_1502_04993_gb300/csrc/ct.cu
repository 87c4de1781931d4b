// Continuous-time form (Sec. 2.3, Eq. 8-14): spike times off any grid, one uniform delay d (Sec. 2.4).
//
// The recording [t_begin, t_end) is cut at every distinct arrival time t_jk + d and every spike time into
// columns: column 0 starts at t_begin, column m covers [c_m, c_{m+1}) and the last one ends at t_end.  On
// the columns the path is the grid path with one decay per column instead of one constant a:
//   v_j(c_{m+1}) = a_m v_j(c_m) + (arrivals of j at c_{m+1}),  a_m = exp(-(c_{m+1} - c_m) / tau)   (Eq. 13)
//   U_i(c_m) = b_i + (W v)_i(c_m)                                                                  (Eq. 3, 8)
//   the integral of e^{U_i} over column m and its weight in dL/dW: ct_link.cuh                   (Eq. 10, 14)
//   the spike part: U at the spike columns (a spike at c_m sees the arrivals at c_m, H(0) = 1).
//
// Set-up (once per problem, on the device): the spike and arrival events are bucketed by time, every bucket
// sorted, equal times merged into one column; each spike learns its column (the spike list of the U
// epilogue and the raster) and each arrival the column before its own (the source list of the filter,
// whose recursion adds S[t - 1] at t).  Per tau: the column constants and the segment decays.
#include <algorithm>
#include <cmath>
#include <vector>

#include "ct_link.cuh"
#include "glm_internal.h"

namespace glm {

namespace {

struct CtItem {
    double t;
    int32_t g;   // index of the spike in the CSR arrays
    int32_t jk;  // row << 1 | kind (0: the spike itself, 1: its arrival)
};

struct CtBuild {
    int32_t n;
    int64_t q;
    double t_begin, t_end, delay, inv_h;
    int64_t nb;  // time buckets
    const int64_t* offs;
    const double* times;
    int32_t* cnt;    // [nb] counts, then fill cursors
    int32_t* start;  // [nb + 1] exclusive prefix of the counts
    CtItem* items;
};

__device__ __forceinline__ int64_t bucket_of(const CtBuild& B, double t) {
    const int64_t k = (int64_t)((t - B.t_begin) * B.inv_h);  // t >= t_begin
    return k < B.nb ? k : B.nb - 1;
}

// the row holding spike g: offs[r] <= g < offs[r + 1]
__device__ __forceinline__ int32_t row_of(const int64_t* __restrict__ offs, int32_t n, int64_t g) {
    int32_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const int32_t mid = (lo + hi) >> 1;
        if (offs[mid] <= g)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

__global__ void ct_count_kernel(const __grid_constant__ CtBuild B) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < B.q; g += (int64_t)gridDim.x * blockDim.x) {
        const double t = B.times[g];
        atomicAdd(B.cnt + bucket_of(B, t), 1);
        const double e = t + B.delay;
        if (e < B.t_end) atomicAdd(B.cnt + bucket_of(B, e), 1);
    }
}

__global__ void ct_scatter_kernel(const __grid_constant__ CtBuild B) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < B.q; g += (int64_t)gridDim.x * blockDim.x) {
        const int32_t j = row_of(B.offs, B.n, g);
        const double t = B.times[g];
        int64_t k = bucket_of(B, t);
        B.items[B.start[k] + atomicAdd(B.cnt + k, 1)] = CtItem{t, (int32_t)g, j << 1};
        const double e = t + B.delay;
        if (e < B.t_end) {
            k = bucket_of(B, e);
            B.items[B.start[k] + atomicAdd(B.cnt + k, 1)] = CtItem{e, (int32_t)g, (j << 1) | 1};
        }
    }
}

__device__ __forceinline__ bool item_less(const CtItem& x, const CtItem& y) {
    if (x.t != y.t) return x.t < y.t;
    if (x.jk != y.jk) return x.jk < y.jk;
    return x.g < y.g;
}

// Thread per bucket: Shell sort with Ciura's gaps (extended by x2.25), a total order on (t, row, kind,
// spike), so the result does not depend on the order of the atomic fills.
__global__ void ct_sort_kernel(const __grid_constant__ CtBuild B) {
    const int32_t gaps[] = {1, 4, 10, 23, 57, 132, 301, 701, 1577, 3548, 7983, 17961, 40412, 90927, 204585,
                            460316, 1035711, 2330349, 5243285, 11797391};
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < B.nb; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t lo = B.start[k], hi = B.start[k + 1], len = hi - lo;
        if (len < 2) continue;
        int gi = 0;
        while (gi + 1 < 20 && gaps[gi + 1] < len) ++gi;
        for (; gi >= 0; --gi) {
            const int64_t gap = gaps[gi];
            for (int64_t i = lo + gap; i < hi; ++i) {
                const CtItem x = B.items[i];
                int64_t p = i;
                while (p - gap >= lo && item_less(x, B.items[p - gap])) {
                    B.items[p] = B.items[p - gap];
                    p -= gap;
                }
                B.items[p] = x;
            }
        }
    }
}

__global__ void ct_flag_kernel(const CtItem* __restrict__ items, int64_t m, int32_t* __restrict__ flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = (i == 0 || items[i].t != items[i - 1].t) ? 1 : 0;
}

// Column of every item (excl + flag, column 0 being t_begin), the column start times, each spike's
// column and each arrival's source column (its own column - 1).
__global__ void ct_assign_kernel(const CtItem* __restrict__ items, int64_t m, const int32_t* __restrict__ excl,
                                 const int32_t* __restrict__ flag, const int64_t* __restrict__ offs,
                                 const int64_t* __restrict__ aoffs, double* __restrict__ ctime,
                                 int32_t* __restrict__ sp_col, int32_t* __restrict__ a_src) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const CtItem it = items[i];
        const int32_t col = excl[i] + flag[i];
        if (flag[i]) ctime[col] = it.t;
        const int32_t j = it.jk >> 1;
        if (it.jk & 1)
            a_src[aoffs[j] + (it.g - offs[j])] = col - 1;
        else
            sp_col[it.g] = col;
    }
}

__global__ void ct_edges_kernel(double* __restrict__ ctime, int64_t M, int64_t Tpad, double t_begin, double t_end) {
    for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m <= Tpad; m += (int64_t)gridDim.x * blockDim.x) {
        if (m == 0)
            ctime[0] = t_begin;
        else if (m >= M)
            ctime[m] = t_end;
    }
}

__global__ void ct_span_kernel(const double* __restrict__ ctime, int64_t nseg, double* __restrict__ span) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nseg; s += (int64_t)gridDim.x * blockDim.x)
        span[s] = ctime[(s + 1) * SEG] - ctime[s * SEG];
}

// Per tau: column constants (a, 1 - a, one-panel quadrature factors) and the decay over each segment.
__global__ void ct_consts_kernel(const double* __restrict__ ctime, int64_t Tpad, int64_t nseg, double tau,
                                 float* __restrict__ col_a, float4* __restrict__ colc, double* __restrict__ seg_mul) {
    for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < Tpad; m += (int64_t)gridDim.x * blockDim.x) {
        float k[8];
        ct_column(ctime[m + 1] - ctime[m], tau, k);
        col_a[m] = k[0];
        colc[2 * m] = make_float4(k[0], k[1], k[2], k[3]);
        colc[2 * m + 1] = make_float4(k[4], k[5], k[6], k[7]);
        if (m < nseg) seg_mul[m] = exp(-(ctime[(m + 1) * SEG] - ctime[m * SEG]) / tau);
    }
}

// ---- exclusive prefix sum of int32 (three passes: block sums, their scan, apply) ----
constexpr int SCAN_T = 256, SCAN_PER = 4, SCAN_BLK = SCAN_T * SCAN_PER;

__device__ __forceinline__ int32_t block_excl_scan(int32_t v, int32_t* total) {
    __shared__ int32_t ws[SCAN_T / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int32_t o = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += o;
    }
    if (lane == 31) ws[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int32_t y = lane < SCAN_T / 32 ? ws[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int32_t o = __shfl_up_sync(0xffffffffu, y, d);
            if (lane >= d) y += o;
        }
        if (lane < SCAN_T / 32) ws[lane] = y;
    }
    __syncthreads();
    const int32_t before = (wid > 0 ? ws[wid - 1] : 0) + x - v;
    *total = ws[SCAN_T / 32 - 1];
    __syncthreads();
    return before;
}

__global__ void scan_sums_kernel(const int32_t* __restrict__ in, int64_t n, int32_t* __restrict__ bsum) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_BLK + threadIdx.x * SCAN_PER;
    int32_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_PER; ++k)
        if (base + k < n) s += in[base + k];
    int32_t tot;
    block_excl_scan(s, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// one block: bsum <- exclusive prefix of bsum
__global__ void scan_carry_kernel(int32_t* __restrict__ bsum, int64_t nb) {
    int32_t carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += SCAN_T) {
        const int64_t i = b0 + threadIdx.x;
        const int32_t v = i < nb ? bsum[i] : 0;
        int32_t tot;
        const int32_t ex = block_excl_scan(v, &tot);
        if (i < nb) bsum[i] = carry + ex;
        carry += tot;
    }
}

__global__ void scan_apply_kernel(const int32_t* __restrict__ in, int64_t n, const int32_t* __restrict__ bsum,
                                  int32_t* __restrict__ out) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_BLK + threadIdx.x * SCAN_PER;
    int32_t v[SCAN_PER], s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_PER; ++k) {
        v[k] = base + k < n ? in[base + k] : 0;
        s += v[k];
    }
    int32_t tot;
    int32_t run = bsum[blockIdx.x] + block_excl_scan(s, &tot);
#pragma unroll
    for (int k = 0; k < SCAN_PER; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
}

// out[i] = sum_{k < i} in[k]; scratch holds ceil(n / 1024) ints
cudaError_t exclusive_scan(const int32_t* in, int32_t* out, int64_t n, int32_t* scratch, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int64_t nb = (n + SCAN_BLK - 1) / SCAN_BLK;
    scan_sums_kernel<<<(unsigned)nb, SCAN_T, 0, st>>>(in, n, scratch);
    scan_carry_kernel<<<1, SCAN_T, 0, st>>>(scratch, nb);
    scan_apply_kernel<<<(unsigned)nb, SCAN_T, 0, st>>>(in, n, scratch, out);
    return cudaGetLastError();
}

unsigned grid_for(int64_t work, int sms) {
    const int64_t g = (work + 255) / 256;
    const int64_t cap = (int64_t)sms * 16;
    return (unsigned)std::max<int64_t>(1, std::min(g, cap));
}

}  // namespace

// Columns of a continuous-time problem.  offs/times: device copies of the CSR spike times; qa arrivals
// (row j's arrivals are its spikes with t + delay < t_end, a prefix of the row).  On success *M is the
// number of columns and *items / *excl / *flag hold the sorted events for ct_finish_columns (device memory
// the caller frees with cudaFree).
int ct_build_columns(glm_ctx* c, int32_t n, int64_t q, int64_t qa, double t_begin, double t_end, double delay,
                     const int64_t* offs, const double* times, int64_t* M, void** items_out, int32_t** excl_out,
                     int32_t** flag_out) {
    const int64_t m = q + qa;  // events
    *M = 1;
    *items_out = nullptr;
    *excl_out = *flag_out = nullptr;
    if (m == 0) return GLM_OK;
    CtBuild B;
    B.n = n;
    B.q = q;
    B.t_begin = t_begin;
    B.t_end = t_end;
    B.delay = delay;
    B.nb = std::max<int64_t>(1, m / 4);
    B.inv_h = (double)B.nb / (t_end - t_begin);
    B.offs = offs;
    B.times = times;
    const int64_t nbs = (B.nb + 1 + SCAN_BLK - 1) / SCAN_BLK + (m + SCAN_BLK - 1) / SCAN_BLK + 2;
    CtItem* items = nullptr;
    int32_t *cnt = nullptr, *start = nullptr, *flag = nullptr, *excl = nullptr, *scratch = nullptr;
    auto cleanup = [&](int rc) {
        cudaFree(cnt);
        cudaFree(start);
        cudaFree(scratch);
        if (rc) {
            cudaFree(items);
            cudaFree(flag);
            cudaFree(excl);
        }
        return rc;
    };
    if (cudaMalloc(&items, sizeof(CtItem) * m) != cudaSuccess || cudaMalloc(&cnt, sizeof(int32_t) * (B.nb + 1)) != cudaSuccess ||
        cudaMalloc(&start, sizeof(int32_t) * (B.nb + 1)) != cudaSuccess ||
        cudaMalloc(&flag, sizeof(int32_t) * m) != cudaSuccess || cudaMalloc(&excl, sizeof(int32_t) * m) != cudaSuccess ||
        cudaMalloc(&scratch, sizeof(int32_t) * nbs) != cudaSuccess) {
        cudaGetLastError();
        return cleanup(set_error(c, GLM_ERR_OOM, "continuous-time set-up buffers"));
    }
    cudaStream_t st = c->stream;
    B.cnt = cnt;
    B.start = start;
    B.items = items;
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (B.nb + 1), st);
    if (e == cudaSuccess) {
        ct_count_kernel<<<grid_for(q, c->sm_count), 256, 0, st>>>(B);
        e = exclusive_scan(cnt, start, B.nb + 1, scratch, st);  // start[nb] = events counted
    }
    // the device's event count must be the host's before any item is placed
    int32_t counted = -1;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&counted, start + B.nb, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && counted != (int32_t)m) {
        c->launches += 4;
        return cleanup(set_error(c, GLM_ERR_INVALID_ARG, "event count differs between host and device"));
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * B.nb, st);
    if (e == cudaSuccess) {
        ct_scatter_kernel<<<grid_for(q, c->sm_count), 256, 0, st>>>(B);
        ct_sort_kernel<<<grid_for(B.nb, c->sm_count), 256, 0, st>>>(B);
        ct_flag_kernel<<<grid_for(m, c->sm_count), 256, 0, st>>>(items, m, flag);
        e = exclusive_scan(flag, excl, m, scratch, st);
    }
    int32_t last[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&last[0], excl + m - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&last[1], flag + m - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    c->launches += 10;
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cleanup(set_error(c, GLM_ERR_CUDA, cudaGetErrorString(e)));
    }
    *M = 1 + (int64_t)last[0] + last[1];
    *items_out = items;
    *excl_out = excl;
    *flag_out = flag;
    return cleanup(GLM_OK);
}

cudaError_t ct_finish_columns(glm_ctx* c, const void* items, const int32_t* excl, const int32_t* flag, int64_t m) {
    const Problem& P = c->pb;
    Buffers& B = c->buf;
    cudaStream_t st = c->stream;
    ct_edges_kernel<<<grid_for(P.Tpad + 1, c->sm_count), 256, 0, st>>>(B.ctime, P.T, P.Tpad, P.t_begin, P.t_end);
    if (m > 0)
        ct_assign_kernel<<<grid_for(m, c->sm_count), 256, 0, st>>>(static_cast<const CtItem*>(items), m, excl, flag,
                                                                   B.offs, B.aoffs, B.ctime, B.bins, B.abins);
    ct_span_kernel<<<grid_for(P.nseg, c->sm_count), 256, 0, st>>>(B.ctime, P.nseg, B.tile_span);
    c->launches += m > 0 ? 3 : 2;
    return cudaGetLastError();
}

cudaError_t launch_ct_consts(glm_ctx* c) {
    const Problem& P = c->pb;
    Buffers& B = c->buf;
    ct_consts_kernel<<<grid_for(P.Tpad, c->sm_count), 256, 0, c->stream>>>(
        B.ctime, P.Tpad, P.nseg, P.tau, B.col_a, reinterpret_cast<float4*>(B.colc), B.seg_mul);
    return cudaGetLastError();
}

}  // namespace glm

extern "C" int glm_ct_interval(double u, double D, double tau, double* F, double* G) {
    if (!(D >= 0) || !(tau > 0) || !std::isfinite(u) || !std::isfinite(D) || !std::isfinite(tau) || !F || !G)
        return GLM_ERR_INVALID_ARG;
    float col[8];
    glm::ct_column(D, tau, col);
    float dF = 0.f, eg = 0.f;
    glm::ct_link((float)u, col, (float)tau, &dF, &eg);
    *F = D + (double)dF;
    *G = tau * (double)eg;
    return GLM_OK;
}

// dF/dtau at fixed u for one column (ct_dtau), on the host, by the same FP32 code as the epilogue.
extern "C" int glm_ct_interval_dtau(double u, double D, double tau, double* dFdtau) {
    if (!(D >= 0) || !(tau > 0) || !std::isfinite(u) || !std::isfinite(D) || !std::isfinite(tau) || !dFdtau)
        return GLM_ERR_INVALID_ARG;
    float col[8];
    glm::ct_column(D, tau, col);
    float dF = 0.f, eg = 0.f;
    glm::ct_link((float)u, col, (float)tau, &dF, &eg);
    *dFdtau = (double)glm::ct_dtau((float)u, col[0], col[1], (float)tau, dF);
    return GLM_OK;
}
