// The plain FP32 form of the two contractions (CUDA cores, no tensor cores):
//   step a3/a4:  U = b 1^T + W X (Eq. 3) with the link applied in the epilogue (Eq. 5):
//                E[i][t] = dt exp(U_i[t]) stored FP32, per (bin tile, row) FP64 sums of exp(U).  The
//                spike-time term of Eq. 7 is not taken from this U: the FP32 form forms it in the row
//                reduction as q_i b_i + sum_j W_ij C_ij from the FP64 spike term C, because the rounding of
//                U's FP32 accumulation, summed over the spike bins, alone comes to ~1e-9 of L
//   step a5:     P_s = E X^T over a split s of the bins (FP32, two-level accumulation)
// 128 x 128 output tiles, 256 threads, 8 x 8 outputs per thread, operands staged in shared memory.
#include <cmath>

#include "expm1_acc.cuh"
#include "glm_internal.h"

namespace glm {

constexpr int SB = 128;   // tile edge
constexpr int SK = 16;    // k step
constexpr int ST = 256;   // threads
constexpr int G_INNER = 1024;  // bins accumulated in the inner FP32 sum of the gradient product
// row stride (floats) of the operand tiles in shared memory: 16-byte aligned rows, and the transposing
// stores of four k-rows by one warp fall into two banks per address group instead of four
constexpr int SBP = SB + 4;

int simt_tile_t() { return SB; }

struct SimtUArgs {
    int32_t n;
    int64_t T, Tpad;
    double dt;
    const float* W;   // [n][n]
    const float* b;   // [n]
    const double* eb; // [n]  exp(b_i) in FP64
    const float* X;   // [n][Tpad]
    float* E;         // [n][Tpad]
    double* part_e;   // [n][ntile]
    int64_t ntile;    // bin tiles, Tpad / 128
    int* flags;
    const int32_t* rows;  // evaluated rows (null: all n); tile row l is row rows[l] for l < m
    int32_t m;
};

__device__ __forceinline__ int32_t row_of(const SimtUArgs& A, int32_t l) {
    return l < A.m ? (A.rows ? A.rows[l] : l) : A.n;
}

// 4-byte asynchronous copy global -> shared (cp.async); pred false fills zeros and reads nothing
__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool pred) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(src), "r"(pred ? 4 : 0) : "memory");
}
// 16-byte asynchronous copy (both addresses 16-byte aligned), through L2 only
__device__ __forceinline__ void cp_async16(float* dst, const float* src, bool pred) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(src), "r"(pred ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// U tile rows i0..i0+127 (of the evaluated rows), bins t0..t0+127.  A = W (row-major, K contiguous), B = X (K x N, N contiguous).
// Blocks run row tile fastest (block id = bin tile * mt + row tile): the row tiles of one bin tile read the
// same X tile while it is in L2.  Two-level sum: the products of two k-steps (32 sources) go into a
// register tile sum, which is added to the thread's column of totals in shared memory.  With both levels
// in registers the kernel needed over 200 registers and ran one block (eight warps) per SM; with the totals
// in shared memory two blocks fit, and their sixteen warps hide the shared-memory latency of the inner
// loop.  The epilogue runs as a rolled loop over rows staged in shared memory: fully unrolled, the k-tile
// body and the 64 inlined exponentials of the epilogue outgrew the instruction cache.
constexpr int EPI_LD = SB + 4;  // row stride of the epilogue staging (floats): 16-byte rows, fewer bank conflicts
constexpr int U_FLUSH = 2;      // k-steps per register tile sum
constexpr size_t U_SMEM = (size_t)(4 * SK * SBP + 64 * ST) * sizeof(float);
static_assert(4 * SK * SBP >= 64 * EPI_LD, "the epilogue staging reuses the operand tiles");
__global__ void __launch_bounds__(ST, 2) simt_u_kernel(const __grid_constant__ SimtUArgs A) {
    // operands: As[2][SK][SBP] then Bs[2][SK][SBP] (after the k loop the same memory stages 64 rows of U);
    // then the totals, [64][ST]: element r * 8 + c of thread tid at [(r * 8 + c) * ST + tid]
    extern __shared__ __align__(16) float sm[];
    auto As = reinterpret_cast<float(*)[SK][SBP]>(sm);
    auto Bs = reinterpret_cast<float(*)[SK][SBP]>(sm + 2 * SK * SBP);
    float* tot = sm + 4 * SK * SBP;
    const int tid = threadIdx.x;
    // thread (ty, tx) owns rows ty*4.. and 64+ty*4.., columns tx*4.. and 64+tx*4..; a warp spans 4 ty x 8 tx,
    // so each of its four 16-byte operand loads per k covers 64 or 128 contiguous bytes: one wavefront
    const int tx = ((tid >> 5) & 1) * 8 + (tid & 7), ty = (tid >> 6) * 4 + ((tid >> 3) & 3);
    const int32_t mt = (A.m + SB - 1) / SB;
    const int32_t i0 = (int32_t)(blockIdx.x % mt) * SB;
    const int64_t bt = (int64_t)(blockIdx.x / mt);
    const int64_t t0 = bt * SB;
    const int32_t n = A.n;
    // loader mapping
    const int a_row = tid >> 2, a_col = (tid & 3) * 4;  // rows a_row and a_row + 64, k a_col..+3
    const int b_row = tid >> 5, b_col = (tid & 31) * 4; // k rows b_row and b_row + 8, bins b_col..+3
    // operand tiles by asynchronous copies issued one k-step ahead (no staging registers): W transposed
    // into [k][row] 4 bytes at a time, X rows 16 bytes at a time; zeros past n
    auto load = [&](int k0, int buf) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int32_t i = row_of(A, i0 + a_row + 64 * h);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int32_t k = k0 + a_col + q;
                const bool ok = i < n && k < n;
                cp_async4(&As[buf][a_col + q][a_row + 64 * h], A.W + (ok ? (int64_t)i * n + k : 0), ok);
            }
            const int32_t kb = k0 + b_row + 8 * h;
            cp_async16(&Bs[buf][b_row + 8 * h][b_col], A.X + (kb < n ? (int64_t)kb * A.Tpad + t0 + b_col : 0), kb < n);
        }
        cp_async_commit();
    };
    const int nk = (n + SK - 1) / SK;
#pragma unroll
    for (int e = 0; e < 64; ++e) tot[e * ST + tid] = 0.f;
    load(0, 0);
    cp_async_wait_all();
    __syncthreads();
    // Two-level accumulation: a single running FP32 sum over ~1000 sources drops the many small terms
    // (sources whose filtered train has decayed) below half an ulp of the total, and since most inputs are
    // excitatory those losses have one sign: at N = 1000 the mean of U came out ~2e-8 low, ~1.4e-8 of L.
    // Tile sums of 32 terms keep those terms.
    float tl[8][8];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) tl[r][c] = 0.f;
    for (int kt = 0; kt < nk; ++kt) {
        const int cur = kt & 1;
        if (kt + 1 < nk) load((kt + 1) * SK, cur ^ 1);
#pragma unroll 4
        for (int k = 0; k < SK; ++k) {
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
        if ((kt + 1) % U_FLUSH == 0 || kt + 1 == nk) {
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    tot[(r * 8 + c) * ST + tid] += tl[r][c];
                    tl[r][c] = 0.f;
                }
        }
        cp_async_wait_all();  // the next k-step's tiles have landed
        __syncthreads();      // ... for every thread, and every thread is done reading this one
    }
    // epilogue.  With v = (W X)_i[t]:  e^{U} = e^{b_i} (1 + expm1(v)).  e^{b_i} comes in FP64 and the
    // integer count of bins is kept apart from the FP32 sum of expm1(v), so the part of the integral that
    // repeats over quiet bins (U ~ b_i) carries no FP32 rounding of exp or of b + v; expm1 is correctly
    // rounded (expm1_acc.cuh), so its rounding carries no bias into the sum either.
    // E = dt e (0 beyond T) in FP32; FP64 row sums of e per tile.  Two halves of 64 rows: the threads
    // stage their v, then each warp takes 8 rows, a lane 4 consecutive bins of a row.
    const int warp = tid >> 5, lane = tid & 31;
    bool bad = false;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        // the k loop's last barrier (or the previous half's) has passed: the staging memory is free
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) {
            float* dst = sm + (ty * 4 + rr) * EPI_LD;
            const float* v = tot + ((4 * half + rr) * 8) * ST + tid;
            *reinterpret_cast<float4*>(dst + tx * 4) = make_float4(v[0], v[ST], v[2 * ST], v[3 * ST]);
            *reinterpret_cast<float4*>(dst + 64 + tx * 4) = make_float4(v[4 * ST], v[5 * ST], v[6 * ST], v[7 * ST]);
        }
        __syncthreads();
#pragma unroll 1
        for (int j = 0; j < 8; ++j) {
            const int lr = warp * 8 + j;  // row within the half
            const int32_t i = row_of(A, i0 + 64 * half + lr);
            const double ebi = (i < n) ? A.eb[i] : 0.0;
            const float sh = (i < n) ? fminf(A.b[i] - EXP_SPLIT_FLOOR, 0.f) : 0.f;  // U - c = v + sh
            const float dteb = (float)(A.dt * ebi);
            const float4 v = *reinterpret_cast<const float4*>(sm + lr * EPI_LD + lane * 4);
            const float vv[4] = {v.x, v.y, v.z, v.w};
            float ev[4];
            float msum = 0.f;
            int cnt = 0;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int64_t t = t0 + lane * 4 + c;
                const float m = expm1_acc(vv[c] + sh);
                const bool valid = t < A.T;
                bad |= valid && !(m <= 3.0e38f);
                if (valid) {
                    msum += m;
                    ++cnt;
                }
                ev[c] = valid ? fmaf(dteb, m, dteb) : 0.f;
            }
            double rs = ebi * ((double)cnt + (double)msum);
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) rs += __shfl_xor_sync(0xffffffffu, rs, off);
            if (i < n) {
                *reinterpret_cast<float4*>(A.E + (int64_t)i * A.Tpad + t0 + lane * 4) = make_float4(ev[0], ev[1], ev[2], ev[3]);
                if (lane == 0) A.part_e[(int64_t)i * A.ntile + bt] = rs;
            }
        }
        __syncthreads();
    }
    if (bad) atomicOr(A.flags, 1);
}

struct SimtGArgs {
    int32_t n;
    int64_t Tpad;
    int64_t k_per_split;
    const float* E;   // [n][Tpad]
    const float* X;   // [n][Tpad]
    float* part_g;    // [nsplit][n][n]
};

// part_g[s][i][j] = sum over bins of split s of E[i][t] X[j][t].  Both operands K contiguous; they are
// transposed into shared memory ([k][row]) by 4-byte asynchronous copies issued one k-step ahead, so the
// loads neither hold registers nor stall the products (with register staging the long-scoreboard wait on
// the loads was the largest stall).  Inner k loop as in simt_u_kernel.  The outer level of the two-level
// sum (every G_INNER bins) lives in shared memory, one column per thread: with it in registers the kernel
// needed 191 registers and ran one block per SM, whose eight warps could not hide the shared-memory
// latency of the inner loop; without, two blocks fit.
constexpr size_t G_SMEM = (size_t)(4 * SK * SBP + 64 * ST) * sizeof(float);
__global__ void __launch_bounds__(ST, 2) simt_grad_kernel(const __grid_constant__ SimtGArgs A) {
    extern __shared__ __align__(16) float gsm[];
    auto As = reinterpret_cast<float(*)[SK][SBP]>(gsm);
    auto Bs = reinterpret_cast<float(*)[SK][SBP]>(gsm + 2 * SK * SBP);
    float* tot = gsm + 4 * SK * SBP;  // [64][ST]: element r * 8 + c of thread tid at [(r * 8 + c) * ST + tid]
    const int tid = threadIdx.x;
    // thread (ty, tx) owns rows ty*4.. and 64+ty*4.., columns tx*4.. and 64+tx*4..; a warp spans 4 ty x 8 tx,
    // so each of its four 16-byte operand loads per k covers 64 or 128 contiguous bytes: one wavefront
    const int tx = ((tid >> 5) & 1) * 8 + (tid & 7), ty = (tid >> 6) * 4 + ((tid >> 3) & 3);
    const int32_t i0 = blockIdx.y * SB, j0 = blockIdx.x * SB;
    const int64_t kb = (int64_t)blockIdx.z * A.k_per_split;
    const int64_t ke = min(kb + A.k_per_split, A.Tpad);
    const int32_t n = A.n;
    float acc[8][8];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            acc[r][c] = 0.f;
            tot[(r * 8 + c) * ST + tid] = 0.f;
        }
    const int l_row = tid >> 2, l_col = (tid & 3) * 4;  // rows l_row, l_row + 64; k l_col..+3
    auto load = [&](int64_t k0, int buf) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int r = l_row + 64 * h;
            const int32_t i = i0 + r, j = j0 + r;
            const float* e = A.E + (int64_t)(i < n ? i : 0) * A.Tpad + k0 + l_col;
            const float* x = A.X + (int64_t)(j < n ? j : 0) * A.Tpad + k0 + l_col;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                cp_async4(&As[buf][l_col + q][r], e + q, i < n);
                cp_async4(&Bs[buf][l_col + q][r], x + q, j < n);
            }
        }
        cp_async_commit();
    };
    if (kb < ke) load(kb, 0);
    cp_async_wait_all();
    __syncthreads();
    int64_t since = 0;
    for (int64_t k0 = kb; k0 < ke; k0 += SK) {
        const int cur = (int)(((k0 - kb) / SK) & 1);
        if (k0 + SK < ke) load(k0 + SK, cur ^ 1);
        float4 a0 = *reinterpret_cast<const float4*>(&As[cur][0][ty * 4]);
        float4 a1 = *reinterpret_cast<const float4*>(&As[cur][0][64 + ty * 4]);
        float4 b0 = *reinterpret_cast<const float4*>(&Bs[cur][0][tx * 4]);
        float4 b1 = *reinterpret_cast<const float4*>(&Bs[cur][0][64 + tx * 4]);
#pragma unroll 4
        for (int k = 0; k < SK; ++k) {
            const int kn = (k + 1 < SK) ? k + 1 : k;
            const float4 na0 = *reinterpret_cast<const float4*>(&As[cur][kn][ty * 4]);
            const float4 na1 = *reinterpret_cast<const float4*>(&As[cur][kn][64 + ty * 4]);
            const float4 nb0 = *reinterpret_cast<const float4*>(&Bs[cur][kn][tx * 4]);
            const float4 nb1 = *reinterpret_cast<const float4*>(&Bs[cur][kn][64 + tx * 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(av[r], bv[c], acc[r][c]);
            a0 = na0;
            a1 = na1;
            b0 = nb0;
            b1 = nb1;
        }
        since += SK;
        if (since == G_INNER) {
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    tot[(r * 8 + c) * ST + tid] += acc[r][c];
                    acc[r][c] = 0.f;
                }
            since = 0;
        }
        cp_async_wait_all();  // the next k-step's tiles have landed
        __syncthreads();      // ... for every thread, and every thread is done reading this one
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int32_t i = i0 + (r < 4 ? ty * 4 + r : 64 + ty * 4 + (r - 4));
        if (i >= n) continue;
        float* dst = A.part_g + ((int64_t)blockIdx.z * n + i) * n;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int32_t j = j0 + (c < 4 ? tx * 4 + c : 64 + tx * 4 + (c - 4));
            if (j < n) dst[j] = tot[(r * 8 + c) * ST + tid] + acc[r][c];
        }
    }
}

int grad_nsplit(const glm_ctx* c) {
    const int64_t tiles = (int64_t)((c->pb.n + SB - 1) / SB) * ((c->pb.n + SB - 1) / SB);
    int64_t s = (4 * (int64_t)c->sm_count + tiles - 1) / tiles;
    const int64_t kmax = c->pb.Tpad / SK;
    if (s > kmax) s = kmax;
    if (s < 1) s = 1;
    if (s > 256) s = 256;
    return (int)s;
}

// exp(b_i) in FP64 for the epilogue; flags non-finite b
__global__ void exp_bias_kernel(int32_t n, const float* __restrict__ b, double* __restrict__ eb, int* flags) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = exp((double)fmaxf(b[i], EXP_SPLIT_FLOOR));
    if (!isfinite(b[i]) || !(v <= 1e300)) atomicOr(flags, 1);
    eb[i] = v;
}

void launch_exp_bias(glm_ctx* c, const float* b) {
    exp_bias_kernel<<<(c->pb.n + 255) / 256, 256, 0, c->stream>>>(c->pb.n, b, c->buf.eb, c->buf.flags);
}

cudaError_t launch_simt_u_epilogue(glm_ctx* c, const float* W, const float* b, const int32_t* rows, int32_t m) {
    const Problem& P = c->pb;
    launch_exp_bias(c, b);
    SimtUArgs A;
    A.n = P.n;
    A.T = P.T;
    A.Tpad = P.Tpad;
    A.dt = P.dt;
    A.W = W;
    A.b = b;
    A.eb = c->buf.eb;
    A.X = reinterpret_cast<const float*>(c->buf.X);
    A.E = reinterpret_cast<float*>(c->buf.E);
    A.part_e = c->buf.part_e;
    A.ntile = P.Tpad / SB;
    A.flags = c->buf.flags;
    A.rows = rows;
    A.m = rows ? m : P.n;
    // one block per (row tile, bin tile), row tiles fastest
    const int64_t blocks = (int64_t)((A.m + SB - 1) / SB) * A.ntile;
    const cudaError_t e = cudaFuncSetAttribute(simt_u_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)U_SMEM);
    if (e != cudaSuccess) return e;
    simt_u_kernel<<<(unsigned)blocks, ST, U_SMEM, c->stream>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_simt_grad(glm_ctx* c) {
    const Problem& P = c->pb;
    const int ns = grad_nsplit(c);
    SimtGArgs A;
    A.n = P.n;
    A.Tpad = P.Tpad;
    int64_t kps = (P.Tpad + ns - 1) / ns;
    kps = ((kps + G_INNER - 1) / G_INNER) * G_INNER;
    A.k_per_split = kps;
    A.E = reinterpret_cast<const float*>(c->buf.E);
    A.X = reinterpret_cast<const float*>(c->buf.X);
    A.part_g = c->buf.part_g;
    dim3 grid((P.n + SB - 1) / SB, (P.n + SB - 1) / SB, ns);
    const cudaError_t e = cudaFuncSetAttribute(simt_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G_SMEM);
    if (e != cudaSuccess) return e;
    simt_grad_kernel<<<grid, ST, G_SMEM, c->stream>>>(A);
    return cudaGetLastError();
}

}  // namespace glm

// The FP32 form's e^v - 1 (expm1_acc.cuh), evaluated on the host by the same code as the epilogue's.
extern "C" int glm_expm1(const float* v_host, int64_t n, float* out_host) {
    if (n < 0 || (n > 0 && (!v_host || !out_host))) return GLM_ERR_INVALID_ARG;
    for (int64_t k = 0; k < n; ++k) out_host[k] = glm::expm1_acc(v_host[k]);
    return GLM_OK;
}
