// Step a7: FP64 reductions in a fixed order (bitwise reproducible).
//   L_i   = q_i b_i + sum_j W_ij C_ij - dt sum_t exp(U_i[t])     (Eq. 7 with the spike term from C)
//   dL/db_i = q_i - dt sum_t exp(U_i[t])                         (Eq. 12, j = 0)
//   dL/dW_ij = C_ij - sum_s P_s[i][j],  P_s = sum_{t in split s} dt exp(U_i[t]) X_j[t]   (Eq. 12)
//   L = sum_i L_i                                                (Eq. 1)
#include "glm_internal.h"

namespace glm {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

struct ReduceArgs {
    int32_t n;
    int64_t ntile;
    double dt;
    const float* W;
    const float* b;
    const double* C;
    const double* qd;
    const double* part_e;  // [n][ntile]
    double* L_rows;
    double* gb;
};

// one warp per row
__global__ void reduce_rows_kernel(const __grid_constant__ ReduceArgs A) {
    const int32_t i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= A.n) return;
    double spk = 0.0;
    for (int32_t j = lane; j < A.n; j += 32) spk += (double)A.W[(int64_t)i * A.n + j] * A.C[(int64_t)i * A.n + j];
    double integ = 0.0;
    const double* pe = A.part_e + (int64_t)i * A.ntile;
    for (int64_t t = lane; t < A.ntile; t += 32) integ += pe[t];
    spk = warp_sum(spk);
    integ = warp_sum(integ);
    if (lane == 0) {
        const double q = A.qd[i];
        A.L_rows[i] = q * (double)A.b[i] + spk - A.dt * integ;
        if (A.gb) A.gb[i] = q - A.dt * integ;
    }
}

__global__ void reduce_grad_kernel(int64_t nn, int nsplit, const double* __restrict__ C,
                                   const float* __restrict__ part_g, double* __restrict__ G) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nn) return;
    double s = 0.0;
    for (int p = 0; p < nsplit; ++p) s += (double)part_g[p * nn + e];
    G[e] = C[e] - s;
}

__global__ void total_kernel(int32_t n, const double* __restrict__ L_rows, double* __restrict__ out) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int32_t i = threadIdx.x; i < n; i += blockDim.x) s += L_rows[i];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) *out = v;
    }
}

cudaError_t launch_reduce(glm_ctx* c, const float* W, const float* b, double* L_rows, double* G, double* gb,
                          bool want_grad, int64_t ntile, int nsplit) {
    const Problem& P = c->pb;
    ReduceArgs A;
    A.n = P.n;
    A.ntile = ntile;
    A.dt = P.dt;
    A.W = W;
    A.b = b;
    A.C = c->buf.C;
    A.qd = c->buf.qd;
    A.part_e = c->buf.part_e;
    A.L_rows = L_rows;
    A.gb = gb;
    reduce_rows_kernel<<<(P.n + 7) / 8, 256, 0, c->stream>>>(A);
    if (want_grad && G) {
        const int64_t nn = (int64_t)P.n * P.n;
        reduce_grad_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, c->stream>>>(nn, nsplit, c->buf.C,
                                                                              c->buf.part_g, G);
    }
    return cudaGetLastError();
}

cudaError_t launch_total(glm_ctx* c, const double* L_rows, double* out1) {
    total_kernel<<<1, 1024, 0, c->stream>>>(c->pb.n, L_rows, out1);
    return cudaGetLastError();
}

}  // namespace glm
