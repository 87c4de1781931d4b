// Step a2: the spike term of the gradient and of the log-likelihood,
//   C_ij = sum_{t : S_i[t] = 1} X_j[t]   (the sum over v_ij(t_ik) in Eq. 12),
// which does not depend on W or b and is computed once per problem (Sec. 2.3.3, 2.6.1).  With it
//   sum_t S_i[t] U_i[t] = q_i b_i + sum_j W_ij C_ij    and    dL_i/dW_ij = C_ij - dt sum_t e^{U_i[t]} X_j[t].
//
// Block = (16 presynaptic rows j, a part of the time axis, a slice of postsynaptic rows i).  For each
// 2048-bin sub-chunk the 16 warps scan X_j for the 16 rows into shared memory (warp = one 256-bin segment
// x 8 rows, started from the FP64 segment carries), then every thread walks the spikes of its rows i in
// the sub-chunk, loading 8 spike bins ahead, and accumulates X_j[t] for the 16 rows.  Sums are kept as an
// FP32 hi + lo pair (TwoSum) refreshed every 8 spikes, so they carry ~44 significant bits, and their
// order is fixed: the result is deterministic.
#include <cmath>

#include "glm_internal.h"
#include "scan_dev.cuh"

namespace glm {

constexpr int ST_THREADS = 512;
constexpr int ST_JB = 16;                     // presynaptic rows per block
constexpr int ST_SUBSEGS = 8;                 // 2048 bins per sub-chunk
constexpr int ST_SUB = ST_SUBSEGS * SEG;
constexpr int ST_KI = 2;                      // postsynaptic rows per thread
constexpr int ST_ROWS_PER_SLICE = ST_THREADS * ST_KI;
constexpr int ST_FLUSH = 8;                   // spikes summed in plain FP32 before a TwoSum
constexpr int ST_BATCH = 8;                   // spike bins loaded ahead per row

// Xs layout: [bin][16 floats] = 4 chunks of 16 bytes per bin, chunk index XOR-swizzled by bin so that the
// phase-A stores (lanes 8 bins apart) spread over the banks.
__device__ __forceinline__ int xs_slot(int bin, int chunk) { return bin * 4 + (chunk ^ ((bin >> 3) & 3)); }

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

__global__ void __launch_bounds__(ST_THREADS, 1) spike_term_kernel(const __grid_constant__ ScanConsts K,
                                                                   const __grid_constant__ SpikeTermArgs A) {
    extern __shared__ float4 Xs[];  // [ST_SUB * 4]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int32_t j0 = blockIdx.x * ST_JB;
    const int64_t part = blockIdx.y;
    const int32_t i_base = blockIdx.z * ST_ROWS_PER_SLICE;
    const float pl_hi = K.pl_hi[lane], pl_lo = K.pl_lo[lane];
    const int64_t sp0 = part * A.segs_per_part;
    const int64_t sp1 = min(sp0 + A.segs_per_part, A.nseg);
    const int seg_w = warp & (ST_SUBSEGS - 1);   // phase A: this warp's segment
    const int half_w = warp >> 3;                // and its 8 of the 16 presynaptic rows

    float acc_hi[ST_KI][ST_JB], acc_lo[ST_KI][ST_JB];
#pragma unroll
    for (int k = 0; k < ST_KI; ++k)
#pragma unroll
        for (int jj = 0; jj < ST_JB; ++jj) acc_hi[k][jj] = acc_lo[k][jj] = 0.f;

    for (int64_t sc = sp0; sc < sp1; sc += ST_SUBSEGS) {
        // ---- phase A: X_j for the 16 rows over this sub-chunk, into shared memory ----
        const int64_t s = sc + seg_w;
        if (s < sp1) {
            const int64_t t0 = s * SEG;
#pragma unroll 1
            for (int pass = 0; pass < 2; ++pass) {  // 4 rows per pass: one 16-byte chunk per bin
                float v[4][8];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int32_t r = j0 + half_w * 8 + pass * 4 + k;
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
                    const int bin = seg_w * SEG + 8 * lane + m;
                    Xs[xs_slot(bin, half_w * 2 + pass)] = make_float4(v[0][m], v[1][m], v[2][m], v[3][m]);
                }
            }
        }
        __syncthreads();
        // ---- phase B: the spikes of this thread's postsynaptic rows in [tb, te) ----
        const int64_t tb = sc * SEG;
        const int64_t sn = min(sp1, sc + ST_SUBSEGS);
#pragma unroll
        for (int k = 0; k < ST_KI; ++k) {
            const int32_t i = i_base + threadIdx.x + k * ST_THREADS;
            if (i >= A.n) continue;
            const int64_t o0 = A.offs[i];
            const int64_t k0 = o0 + A.seg_first[(int64_t)i * A.nseg + sc];
            const int64_t k1 = (sn < A.nseg) ? o0 + A.seg_first[(int64_t)i * A.nseg + sn] : A.offs[i + 1];
            float sh[ST_JB];
#pragma unroll
            for (int jj = 0; jj < ST_JB; ++jj) sh[jj] = 0.f;
            for (int64_t kb = k0; kb < k1; kb += ST_BATCH) {
                int tl[ST_BATCH];
#pragma unroll
                for (int u = 0; u < ST_BATCH; ++u) tl[u] = (kb + u < k1) ? (int)(__ldg(A.bins + kb + u) - tb) : -1;
#pragma unroll
                for (int u = 0; u < ST_BATCH; ++u) {
                    if (tl[u] < 0) break;
#pragma unroll
                    for (int ch = 0; ch < 4; ++ch) {
                        const float4 x = Xs[xs_slot(tl[u], ch)];
                        sh[4 * ch + 0] += x.x;
                        sh[4 * ch + 1] += x.y;
                        sh[4 * ch + 2] += x.z;
                        sh[4 * ch + 3] += x.w;
                    }
                }
                // ST_FLUSH == ST_BATCH: at most 8 values in each plain FP32 sum
#pragma unroll
                for (int jj = 0; jj < ST_JB; ++jj) {
                    two_sum(acc_hi[k][jj], acc_lo[k][jj], sh[jj]);
                    sh[jj] = 0.f;
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < ST_KI; ++k) {
        const int32_t i = i_base + threadIdx.x + k * ST_THREADS;
        if (i >= A.n) continue;
        double* dst = A.C_part + (part * A.n + i) * (int64_t)A.n + j0;
#pragma unroll
        for (int jj = 0; jj < ST_JB; ++jj)
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
    const int64_t groups = (c->pb.n + ST_JB - 1) / ST_JB;
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
    const size_t smem = (size_t)ST_SUB * ST_JB * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(spike_term_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((P.n + ST_JB - 1) / ST_JB, parts, (P.n + ST_ROWS_PER_SLICE - 1) / ST_ROWS_PER_SLICE);
    spike_term_kernel<<<grid, ST_THREADS, smem, c->stream>>>(c->sc, A);
    const int64_t nn = (int64_t)P.n * P.n;
    spike_term_reduce_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, c->stream>>>(nn, parts, c->buf.C_part,
                                                                                c->buf.C);
    return cudaGetLastError();
}

}  // namespace glm
