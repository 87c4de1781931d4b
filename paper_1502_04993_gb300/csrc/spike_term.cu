// Step a2: the spike term of the gradient and of the log-likelihood,
//   C_ij = sum_{t : S_i[t] = 1} X_j[t]   (the sum over v_ij(t_ik) in Eq. 12),
// which does not depend on W or b and is computed once per problem (Sec. 2.3.3, 2.6.1).  With it
//   sum_t S_i[t] U_i[t] = q_i b_i + sum_j W_ij C_ij    and    dL_i/dW_ij = C_ij - dt sum_t e^{U_i[t]} X_j[t].
//
// Block = (8 presynaptic rows j, a part of the time axis, a slice of postsynaptic rows i).  For each
// 4096-bin sub-chunk the 16 warps scan X_j for the 8 rows into shared memory (one 256-bin segment per
// warp, started from the FP64 segment carries), then every thread walks the spikes of its rows i in
// the sub-chunk and accumulates X_j[t].  Sums are kept as an FP32 hi + lo pair (TwoSum) refreshed every
// few spikes, so they carry ~44 significant bits and their order is fixed: the result is deterministic.
#include <cmath>

#include "glm_internal.h"
#include "scan_dev.cuh"

namespace glm {

constexpr int ST_THREADS = 512;
constexpr int ST_SUBSEGS = 16;                // 4096 bins per sub-chunk
constexpr int ST_SUB = ST_SUBSEGS * SEG;
constexpr int ST_KI = 2;                      // postsynaptic rows per thread
constexpr int ST_ROWS_PER_SLICE = ST_THREADS * ST_KI;
constexpr int ST_FLUSH = 4;                   // spikes summed in plain FP32 before a TwoSum

__device__ __forceinline__ int swz(int t) { return t ^ ((t >> 3) & 3); }

__device__ __forceinline__ void two_sum(float& hi, float& lo, float x) {
    const float s = hi + x;
    const float bp = s - hi;
    const float e = (hi - (s - bp)) + (x - bp);
    hi = s;
    lo += e;
}

struct SpikeTermArgs {
    int32_t n;
    int64_t nseg;
    int64_t segs_per_part;
    const int64_t* offs;
    const int32_t* bins;
    const double* seg_carry;
    const int32_t* seg_first;
    double* C_part;  // [parts][n][n]
};

__global__ void __launch_bounds__(ST_THREADS) spike_term_kernel(const __grid_constant__ ScanConsts K,
                                                                const __grid_constant__ SpikeTermArgs A) {
    extern __shared__ float4 smem4[];
    float* Xs = reinterpret_cast<float*>(smem4);  // [ST_SUB][8], bin index swizzled
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int32_t j0 = blockIdx.x * 8;
    const int64_t part = blockIdx.y;
    const int32_t i_base = blockIdx.z * ST_ROWS_PER_SLICE;
    const float pl_hi = K.pl_hi[lane], pl_lo = K.pl_lo[lane];
    const int64_t sp0 = part * A.segs_per_part;
    const int64_t sp1 = min(sp0 + A.segs_per_part, A.nseg);

    float acc_hi[ST_KI][8], acc_lo[ST_KI][8];
#pragma unroll
    for (int k = 0; k < ST_KI; ++k)
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) acc_hi[k][jj] = acc_lo[k][jj] = 0.f;

    for (int64_t sc = sp0; sc < sp1; sc += ST_SUBSEGS) {
        // ---- phase A: X_j for the 8 rows over this sub-chunk ----
        const int64_t s = sc + warp;
        if (warp < ST_SUBSEGS && s < sp1) {
            const int64_t t0 = s * SEG;
            float v[8][8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int32_t r = j0 + k;
                float xs = 0.f;
                uint32_t bits = 0;
                if (r < A.n) {
                    xs = (float)A.seg_carry[(int64_t)r * A.nseg + s];
                    int64_t cur = A.offs[r] + A.seg_first[(int64_t)r * A.nseg + s];
                    bits = seg_bits(A.bins, cur, A.offs[r + 1], t0, lane);
                }
                seg_scan(K, xs, bits, pl_hi, pl_lo, lane, v[k]);
            }
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                const int tloc = warp * SEG + 8 * lane + m;
                float4* dst = reinterpret_cast<float4*>(Xs + (int64_t)swz(tloc) * 8);
                dst[0] = make_float4(v[0][m], v[1][m], v[2][m], v[3][m]);
                dst[1] = make_float4(v[4][m], v[5][m], v[6][m], v[7][m]);
            }
        }
        __syncthreads();
        // ---- phase B: spikes of the postsynaptic rows in this sub-chunk ----
        const int64_t tb = sc * SEG;
        const int64_t te = min(sp1, sc + ST_SUBSEGS) * SEG;
#pragma unroll
        for (int k = 0; k < ST_KI; ++k) {
            const int32_t i = i_base + threadIdx.x + k * ST_THREADS;
            if (i >= A.n) continue;
            // this row's spikes in [tb, te) are bins[k0 .. k1): independent loads, no pointer chase
            const int64_t o0 = A.offs[i];
            const int64_t k0 = o0 + A.seg_first[(int64_t)i * A.nseg + sc];
            const int64_t sn = min(sp1, sc + ST_SUBSEGS);
            const int64_t k1 = (sn < A.nseg) ? o0 + A.seg_first[(int64_t)i * A.nseg + sn] : A.offs[i + 1];
            float sh[8];
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) sh[jj] = 0.f;
            int cnt = 0;
#pragma unroll 4
            for (int64_t kk = k0; kk < k1; ++kk) {
                const int64_t t = __ldg(A.bins + kk);
                const float4* src = reinterpret_cast<const float4*>(Xs + (int64_t)swz((int)(t - tb)) * 8);
                const float4 x0 = src[0], x1 = src[1];
                sh[0] += x0.x; sh[1] += x0.y; sh[2] += x0.z; sh[3] += x0.w;
                sh[4] += x1.x; sh[5] += x1.y; sh[6] += x1.z; sh[7] += x1.w;
                if (++cnt == ST_FLUSH) {
#pragma unroll
                    for (int jj = 0; jj < 8; ++jj) {
                        two_sum(acc_hi[k][jj], acc_lo[k][jj], sh[jj]);
                        sh[jj] = 0.f;
                    }
                    cnt = 0;
                }
            }
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) two_sum(acc_hi[k][jj], acc_lo[k][jj], sh[jj]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < ST_KI; ++k) {
        const int32_t i = i_base + threadIdx.x + k * ST_THREADS;
        if (i >= A.n) continue;
        double* dst = A.C_part + (part * A.n + i) * (int64_t)A.n + j0;
#pragma unroll
        for (int jj = 0; jj < 8; ++jj)
            if (j0 + jj < A.n) dst[jj] = (double)acc_hi[k][jj] + (double)acc_lo[k][jj];
    }
}

// C[i][j] = sum over parts, in part order.
__global__ void spike_term_reduce_kernel(int64_t nn, int parts, const double* __restrict__ C_part,
                                         double* __restrict__ C) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nn) return;
    double s = 0.0;
    for (int p = 0; p < parts; ++p) s += C_part[p * nn + e];
    C[e] = s;
}

int spike_term_parts(const glm_ctx* c) {
    const int64_t nsub = (c->pb.nseg + ST_SUBSEGS - 1) / ST_SUBSEGS;
    const int64_t groups = (c->pb.n + 7) / 8;
    int64_t p = (2 * (int64_t)c->sm_count + groups - 1) / groups;
    if (p < 1) p = 1;
    if (p > nsub) p = nsub;
    if (p > 64) p = 64;
    return (int)p;
}

cudaError_t launch_spike_term(glm_ctx* c) {
    const Problem& P = c->pb;
    const int parts = spike_term_parts(c);
    const int64_t nsub = (P.nseg + ST_SUBSEGS - 1) / ST_SUBSEGS;
    const int64_t subs_per_part = (nsub + parts - 1) / parts;
    SpikeTermArgs A;
    A.n = P.n;
    A.nseg = P.nseg;
    A.segs_per_part = subs_per_part * ST_SUBSEGS;
    A.offs = c->buf.offs;
    A.bins = c->buf.bins;
    A.seg_carry = c->buf.seg_carry;
    A.seg_first = c->buf.seg_first;
    A.C_part = c->buf.C_part;
    const size_t smem = (size_t)ST_SUB * 8 * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(spike_term_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((P.n + 7) / 8, parts, (P.n + ST_ROWS_PER_SLICE - 1) / ST_ROWS_PER_SLICE);
    spike_term_kernel<<<grid, ST_THREADS, smem, c->stream>>>(c->sc, A);
    const int64_t nn = (int64_t)P.n * P.n;
    spike_term_reduce_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, c->stream>>>(nn, parts, c->buf.C_part,
                                                                                c->buf.C);
    return cudaGetLastError();
}

}  // namespace glm
