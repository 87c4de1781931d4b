// glm_loglik_noalloc: the per-row log-likelihood of the plain FP32 form without any device allocation.
//
// Who needs it: callers that may not call cudaMalloc.  Typical cases are processes whose device memory
// is owned by another allocator (a framework's caching pool or a pre-reserved arena that leaves nothing
// for cudaMalloc), and latency-critical loops that must not allocate after start-up (cudaMalloc can
// synchronise the device and fail at run time).  Such a caller passes its own inputs and outputs; the
// only temporary storage this entry point needs lives in one fixed, file-scope device array.
//
// It is a variant of the U-product kernel of simt.cu (128 x 128 tiles, 8 x 8 outputs per thread) that
// keeps its per-(row, tile) partial sums of exp(U) and the values exp(b_i) in that fixed array instead
// of in context memory, skips the store of the rates (no gradient here), and reads X with bounds checks
// so any leading dimension works.  It computes the same quantity as glm_loglik_grad's L_rows.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "expm1_acc.cuh"
#include "glm.h"

namespace {

constexpr int NB = 128;  // tile edge
constexpr int NK = 16;   // k step
constexpr int NT = 256;  // threads
constexpr int MAX_DEVICES = 64;
// e^U = e^c e^(U - c), c = max(b_i, -60): the same split as the library's regular U product
constexpr float NA_EXP_SPLIT_FLOOR = -60.f;

// The fixed scratch: exp(b_i) for i < n, then the partial sums [n][ceil(n_bins / 128)]; every element used
// is written before it is read, so nothing needs clearing between calls.  Every GPU that loads the library
// holds the array until the process exits.
constexpr size_t SCRATCH_DOUBLES = (size_t)GLM_NOALLOC_SCRATCH_BYTES / sizeof(double);
static __device__ __align__(256) double g_scratch[SCRATCH_DOUBLES];

std::mutex g_mu;
void* g_scratch_addr[MAX_DEVICES] = {};

// Device address of g_scratch on the current device (the host-side symbol is only a stand-in).  Looked
// up once per device, on that device's first call.
int scratch_address(double** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        cudaGetLastError();
        return GLM_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return GLM_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = reinterpret_cast<double*>(g_scratch_addr[dev]);
    return GLM_OK;
}

__global__ void na_exp_bias_kernel(int32_t n, const float* __restrict__ b, double* __restrict__ eb) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) eb[i] = exp((double)fmaxf(b[i], NA_EXP_SPLIT_FLOOR));
}

struct NaArgs {
    int32_t n;
    int64_t T, ldx, ntile;
    const float* W;
    const float* X;
    const float* b;
    const double* eb;
    double* part;  // [n][ntile]
};

__global__ void __launch_bounds__(NT) na_u_kernel(const __grid_constant__ NaArgs A) {
    __shared__ __align__(16) float As[2][NK][NB];
    __shared__ __align__(16) float Bs[2][NK][NB];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int32_t i0 = blockIdx.y * NB;
    const int64_t t0 = (int64_t)blockIdx.x * NB;
    const int32_t n = A.n;
    float acc[8][8];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[r][c] = 0.f;
    const int a_row = tid >> 2, a_col = (tid & 3) * 4;
    const int b_row = tid >> 5, b_col = (tid & 31) * 4;
    float ra[2][4], rb[2][4];
    auto load = [&](int k0) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int32_t i = i0 + a_row + 64 * h;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int32_t k = k0 + a_col + q;
                ra[h][q] = (i < n && k < n) ? A.W[(int64_t)i * n + k] : 0.f;
            }
            const int32_t kb = k0 + b_row + 8 * h;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int64_t t = t0 + b_col + q;
                rb[h][q] = (kb < n && t < A.T) ? A.X[(int64_t)kb * A.ldx + t] : 0.f;
            }
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
#pragma unroll
            for (int q = 0; q < 4; ++q) As[buf][a_col + q][a_row + 64 * h] = ra[h][q];
            *reinterpret_cast<float4*>(&Bs[buf][b_row + 8 * h][b_col]) =
                make_float4(rb[h][0], rb[h][1], rb[h][2], rb[h][3]);
        }
    };
    const int nk = (n + NK - 1) / NK;
    load(0);
    store(0);
    __syncthreads();
    // two-level accumulation, as the library's regular FP32 U product does (there over 32 sources): the 16
    // products of each k-step go into a fresh tile sum, added to the total (a single running sum drops small
    // terms with one sign)
    for (int kt = 0; kt < nk; ++kt) {
        const int cur = kt & 1;
        if (kt + 1 < nk) load((kt + 1) * NK);
        float tl[8][8];
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int c = 0; c < 8; ++c) tl[r][c] = 0.f;
#pragma unroll
        for (int k = 0; k < NK; ++k) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[cur][k][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[cur][k][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[cur][k][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[cur][k][64 + tx * 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int c = 0; c < 8; ++c) tl[r][c] = fmaf(av[r], bv[c], tl[r][c]);
        }
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[r][c] += tl[r][c];
        if (kt + 1 < nk) store(cur ^ 1);
        __syncthreads();
    }
    // e^{U} = e^{b_i} (1 + expm1(v)), v = (W X)_i[t]; sums kept as e^{b_i} (count + sum expm1(v)).
    // A non-finite exp or input makes L_i non-finite: that is how it is reported.
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int32_t i = i0 + (r < 4 ? ty * 4 + r : 64 + ty * 4 + (r - 4));
        const double ebi = (i < n) ? A.eb[i] : 0.0;
        float msum = 0.f;
        int cnt = 0;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int64_t t = t0 + (c < 4 ? tx * 4 + c : 64 + tx * 4 + (c - 4));
            const float m = glm::expm1_acc(acc[r][c] + (i < n ? fminf(A.b[i] - NA_EXP_SPLIT_FLOOR, 0.f) : 0.f));
            if (t < A.T) {
                msum += m;
                ++cnt;
            }
        }
        double rs = ebi * ((double)cnt + (double)msum);
#pragma unroll
        for (int off = 8; off >= 1; off >>= 1) rs += __shfl_xor_sync(0xffffffffu, rs, off);
        if (i < n && tx == 0) A.part[(int64_t)i * A.ntile + blockIdx.x] = rs;
    }
}

// L_i = q_i b_i + sum_j W_ij C_ij - dt sum_tiles part[i][tile]   (one warp per row, fixed order)
__global__ void na_rows_kernel(int32_t n, int64_t ntile, double dt, const float* __restrict__ W,
                               const float* __restrict__ b, const double* __restrict__ C,
                               const double* __restrict__ q, const double* __restrict__ part,
                               double* __restrict__ L) {
    const int32_t i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    double spk = 0.0, integ = 0.0;
    for (int32_t j = lane; j < n; j += 32) spk += (double)W[(int64_t)i * n + j] * C[(int64_t)i * n + j];
    for (int64_t t = lane; t < ntile; t += 32) integ += part[(int64_t)i * ntile + t];
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        spk += __shfl_xor_sync(0xffffffffu, spk, off);
        integ += __shfl_xor_sync(0xffffffffu, integ, off);
    }
    if (lane == 0) L[i] = q[i] * (double)b[i] + spk - dt * integ;
}

}  // namespace

extern "C" int glm_loglik_noalloc(int32_t n, int64_t n_bins, double dt, const float* X_dev, int64_t ldx,
                                  const double* C_dev, const double* q_dev, const float* W_dev, const float* b_dev,
                                  double* L_rows_dev, void* cuda_stream) {
    if (n < 1 || n_bins < 1 || ldx < n_bins || !(std::isfinite(dt) && dt > 0) || !X_dev || !C_dev || !q_dev ||
        !W_dev || !b_dev || !L_rows_dev)
        return GLM_ERR_INVALID_ARG;
    const int64_t ntile = (n_bins + NB - 1) / NB;
    // scratch needed: n values of exp(b) and n * ntile partial sums
    if ((double)n * (double)(ntile + 1) > (double)SCRATCH_DOUBLES) return GLM_ERR_SCRATCH_TOO_SMALL;
    double* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    NaArgs A;
    A.n = n;
    A.T = n_bins;
    A.ldx = ldx;
    A.ntile = ntile;
    A.W = W_dev;
    A.X = X_dev;
    A.b = b_dev;
    A.eb = scratch;
    A.part = scratch + n;
    na_exp_bias_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, b_dev, scratch);
    dim3 grid((unsigned)ntile, (unsigned)((n + NB - 1) / NB));
    na_u_kernel<<<grid, NT, 0, st>>>(A);
    na_rows_kernel<<<(n + 7) / 8, 256, 0, st>>>(n, ntile, dt, W_dev, b_dev, C_dev, q_dev, scratch + n, L_rows_dev);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GLM_OK : GLM_ERR_CUDA;
}
