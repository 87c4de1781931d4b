// Step a7: reductions in a fixed order (bitwise reproducible): the per-tile sums in FP64, the FP32 partials of
// the split products as FP32 TwoSum pairs (~48 bits) converted once to FP64.
//   L_i   = sum_{t in sp(i)} U_i[t] - dt sum_t exp(U_i[t])        (Eq. 7), the spike part as
//           q_i b_i + sum over tiles of (sum of U - b at the row's spike bins) from the U-product epilogue in
//           the 16-bit forms (the bias of the tensor cores' FP32 accumulation of U then cancels between the
//           two parts), and in the plain FP32 form as q_i b_i + sum_j W_ij C_ij in FP64 from the exact spike
//           term C (the same sum, since U - b = W X; free of the FP32 rounding of U summed over the spikes)
//   dL/db_i = q_i - dt sum_t exp(U_i[t])                         (Eq. 12, j = 0)
//   dL/dW_ij = C_ij - sum_s P_s[i][j],  P_s = sum_{t in split s} dt exp(U_i[t]) X_j[t]   (Eq. 12)
//   L = sum_i L_i                                                (Eq. 1)
#include <cmath>

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
    const double* C;       // spike term (dL/dW)
    const double* part_s;  // [n][ntile] sums of U - b at the spike bins
    const double* qd;
    const double* part_e;  // [n][ntile]
    int32_t planes;        // planes of part_s and part_e, [planes][n][ntile] (continuous time: CT_PARTS)
    int32_t r0, r1;        // rows outside [r0, r1) (a row range) get L_i = 0 and dL/db_i = 0
    bool spk_from_c;       // spike part q_i b_i + sum_j W_ij C_ij (FP32 form) instead of the part_s sums
    const double* part_self;  // self-delay: [n][ntile] per-tile parts of the diagonal's gradient, or null
    double* gself;            //   their row sums
    double* L_rows;
    double* gb;
};

// one warp per row
__global__ void reduce_rows_kernel(const __grid_constant__ ReduceArgs A) {
    const int32_t i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= A.n) return;
    double spk = 0.0;
    if (A.spk_from_c) {
        const float* Wi = A.W + (int64_t)i * A.n;
        const double* Ci = A.C + (int64_t)i * A.n;
        for (int32_t j = lane; j < A.n; j += 32) spk += (double)Wi[j] * Ci[j];
    } else {
        const double* ps = A.part_s + (int64_t)i * A.ntile;
        for (int64_t t = lane; t < A.ntile; t += 32) spk += ps[t];
    }
    double integ = 0.0;
    const double* pe = A.part_e + (int64_t)i * A.ntile;
    for (int64_t t = lane; t < A.ntile; t += 32) integ += pe[t];
    for (int32_t pl = 1; pl < A.planes; ++pl) {
        const double* ps2 = A.part_s + ((int64_t)pl * A.n + i) * A.ntile;
        const double* pe2 = A.part_e + ((int64_t)pl * A.n + i) * A.ntile;
        for (int64_t t = lane; t < A.ntile; t += 32) {
            if (!A.spk_from_c) spk += ps2[t];
            integ += pe2[t];
        }
    }
    double gs = 0.0;
    if (A.part_self) {
        const double* pq = A.part_self + (int64_t)i * A.ntile;
        for (int64_t t = lane; t < A.ntile; t += 32) gs += pq[t];
        gs = warp_sum(gs);
        if (lane == 0) A.gself[i] = gs;
    }
    spk = warp_sum(spk);
    integ = warp_sum(integ);
    if (lane == 0) {
        const double q = A.qd[i];
        const bool in = i >= A.r0 && i < A.r1;
        A.L_rows[i] = in ? q * (double)A.b[i] + spk - A.dt * integ : 0.0;
        if (A.gb) A.gb[i] = in ? q - A.dt * integ : 0.0;
    }
}

// Sums over the splits p = 0 .. nsplit-1 of part_g[p nn + e], added in split order.  The FP32 partials are
// accumulated as an unevaluated FP32 pair hi + lo with TwoSum (Knuth: hi + err = hi_old + v exactly), which
// keeps ~48 significant bits, and the pair becomes one FP64 value at the end: FP64 arithmetic is a scarce
// pipe on this GPU, and summing the partials in FP64 made these kernels pipe-bound at a tenth of the memory
// bandwidth.  A thread takes 4 consecutive elements (one 16-byte load per split when nn is a multiple of 4,
// so every split plane starts 16-byte aligned), and the loads of 4 splits are issued before their adds.
constexpr int SPLIT_EPT = 4;

__device__ __forceinline__ void two_sum_f(float& hi, float& lo, float v) {
    const float s = hi + v;
    const float bp = s - hi;
    lo += (hi - (s - bp)) + (v - bp);
    hi = s;
}

__device__ __forceinline__ void sum_parts4(const float* __restrict__ part_g, int64_t nn, int64_t e0, int nsplit,
                                           bool vec, double (&out)[SPLIT_EPT]) {
    float hi[SPLIT_EPT], lo[SPLIT_EPT];
#pragma unroll
    for (int i = 0; i < SPLIT_EPT; ++i) hi[i] = lo[i] = 0.f;
    if (vec) {
        int p = 0;
        for (; p + 4 <= nsplit; p += 4) {
            float4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = __ldcs(reinterpret_cast<const float4*>(part_g + (int64_t)(p + u) * nn + e0));
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                two_sum_f(hi[0], lo[0], v[u].x);
                two_sum_f(hi[1], lo[1], v[u].y);
                two_sum_f(hi[2], lo[2], v[u].z);
                two_sum_f(hi[3], lo[3], v[u].w);
            }
        }
        for (; p < nsplit; ++p) {
            const float4 v = __ldcs(reinterpret_cast<const float4*>(part_g + (int64_t)p * nn + e0));
            two_sum_f(hi[0], lo[0], v.x);
            two_sum_f(hi[1], lo[1], v.y);
            two_sum_f(hi[2], lo[2], v.z);
            two_sum_f(hi[3], lo[3], v.w);
        }
    } else {
        for (int p = 0; p < nsplit; ++p)
#pragma unroll
            for (int i = 0; i < SPLIT_EPT; ++i)
                if (e0 + i < nn) two_sum_f(hi[i], lo[i], __ldcs(part_g + (int64_t)p * nn + e0 + i));
    }
#pragma unroll
    for (int i = 0; i < SPLIT_EPT; ++i) out[i] = (double)hi[i] + (double)lo[i];
}

// G rows outside [e0, e1) (element range of a row range) are set to zero
// gself (self-delay, or null): the diagonal element (i, i) also subtracts gself[i] = sum_t dt e^U_i[t] (X_i
// with the self-delay - X_i)[t], which E X^T does not cover
__global__ void reduce_grad_kernel(int64_t nn, int nsplit, const double* __restrict__ C,
                                   const float* __restrict__ part_g, const double* __restrict__ Gacc,
                                   double* __restrict__ G, int64_t e0, int64_t e1, int32_t n,
                                   const double* __restrict__ gself) {
    const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * SPLIT_EPT;
    if (b >= nn) return;
    const bool vec = (nn % SPLIT_EPT) == 0;
    double s[SPLIT_EPT];
    if (b + SPLIT_EPT <= e0 || b >= e1) {  // all outside the row range: no partial sums there
#pragma unroll
        for (int i = 0; i < SPLIT_EPT; ++i)
            if (b + i < nn) G[b + i] = 0.0;
        return;
    }
    if (Gacc) {
#pragma unroll
        for (int i = 0; i < SPLIT_EPT; ++i) s[i] = (b + i < nn) ? Gacc[b + i] : 0.0;
    } else {
        sum_parts4(part_g, nn, b, nsplit, vec, s);
    }
#pragma unroll
    for (int i = 0; i < SPLIT_EPT; ++i) {
        const int64_t e = b + i;
        if (e < nn) {
            double g = (e < e0 || e >= e1) ? 0.0 : C[e] - s[i];
            if (gself && e >= e0 && e < e1 && e / n == e % n) g -= gself[e / n];
            G[e] = g;
        }
    }
}

// C[e] (+)= sum over splits of part_g, in split order.
__global__ void sum_splits_kernel(int64_t nn, int nsplit, const float* __restrict__ part_g, double* __restrict__ C,
                                  bool accumulate) {
    const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * SPLIT_EPT;
    if (b >= nn) return;
    double s[SPLIT_EPT];
    sum_parts4(part_g, nn, b, nsplit, (nn % SPLIT_EPT) == 0, s);
#pragma unroll
    for (int i = 0; i < SPLIT_EPT; ++i)
        if (b + i < nn) C[b + i] = accumulate ? C[b + i] + s[i] : s[i];
}

cudaError_t launch_sum_splits(glm_ctx* c, int nsplit, double* C, bool accumulate) {
    const int64_t nn = (int64_t)c->pb.n * c->pb.n;
    const int64_t threads = (nn + SPLIT_EPT - 1) / SPLIT_EPT;
    sum_splits_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, c->stream>>>(nn, nsplit, c->buf.part_g, C, accumulate);
    return cudaGetLastError();
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

// Row i's share of dL/dtau, up to the factor da/dtau = a dt / tau^2 (applied on the host):
//   r_i = sum_t R_i[t] Z_i[t] = sum_{t in sp(i)} Z_i[t] - dt e^{b_i} sum_t e^{v_i[t]} Z_i[t],
// with Z_i = W_i Y, Y = dX/da on the grid, i.e. Z_i[t] = a Z_i[t-1] + v_i[t-1] (v = U - b).  The epilogue
// left per tile k: P1 = sum e^v a^(t-t0), P2 = sum e^v Z_loc, Zend = Z_loc at the next tile, P3 = sum over
// the spike bins of a^(t-t0), P4 = sum over the spike bins of Z_loc; with Z_start(0) = 0 and
// Z_start(k+1) = A Z_start(k) + Zend(k) (A = a^256) a weight family contributes sum_k Z_start(k) P(k) + P'(k).
// Warp per row: lanes own contiguous tile ranges, a shuffle scan supplies each range's Z_start.
__global__ void tau_rows_kernel(int32_t n, int64_t ntile, double dt, double A256, const double* __restrict__ eb,
                                const double* __restrict__ part_tau, double* __restrict__ rows) {
    const int32_t i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    const int64_t plane = (int64_t)n * ntile;
    const double* p1 = part_tau + (int64_t)i * ntile;
    const double* p2 = p1 + plane;
    const double* ze = p1 + 2 * plane;
    const double* p3 = p1 + 3 * plane;
    const double* p4 = p1 + 4 * plane;
    const int64_t len = (ntile + 31) / 32;
    const int64_t k0 = min((int64_t)lane * len, ntile), k1 = min(k0 + len, ntile);
    // with z = Z_start relative to the range start (0) and w = A^(k - k0):
    double z = 0.0, w = 1.0, Qe = 0.0, Se = 0.0, Qs = 0.0, Ss = 0.0;
    for (int64_t k = k0; k < k1; ++k) {
        Qe = fma(w, p1[k], Qe);
        Se += fma(z, p1[k], p2[k]);
        Qs = fma(w, p3[k], Qs);
        Ss += fma(z, p3[k], p4[k]);
        z = fma(A256, z, ze[k]);
        w *= A256;
    }
    double v = z, m = w;
    for (int d = 1; d < 32; d <<= 1) {
        const double o = __shfl_up_sync(0xffffffffu, v, d), om = __shfl_up_sync(0xffffffffu, m, d);
        if (lane >= d) {
            v = fma(m, o, v);
            m *= om;
        }
    }
    double zin = __shfl_up_sync(0xffffffffu, v, 1);
    if (lane == 0) zin = 0.0;
    double integ = fma(zin, Qe, Se);
    double spk = fma(zin, Qs, Ss);
    integ = warp_sum(integ);
    spk = warp_sum(spk);
    if (lane == 0) rows[i] = spk - dt * eb[i] * integ;
}

// Continuous time: row i's dL/dtau itself, r_i = sum_{spikes} z / tau^2 - e^{c_i} (sum_m e^sh (G_m / tau) z_m /
// tau + sum_m e^sh dF_m/dtau), with z = W y at the column starts (y = tau^2 dv/dtau).  The epilogue left,
// per tile and part of a tile's columns (in column order: tile-major, part-minor), the sums P1, P2, Zend,
// P3, P4, Pex and the part's decay product Aend; with z_start of the first segment 0 (no input before
// t_begin) and z_start(next) = Aend z_start + Zend, a weight family contributes sum z_start P + P'.  The
// chain of segments is cut into contiguous lane ranges as in tau_rows_kernel, each range's own decay
// product composing the shuffle scan.
__global__ void ct_tau_rows_kernel(int32_t n, int64_t ntile, double tau, const double* __restrict__ eb,
                                   const double* __restrict__ part_tau, double* __restrict__ rows) {
    const int32_t i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    const int64_t pl = (int64_t)CT_PARTS * n * ntile;  // one value over all parts, rows and tiles
    const int64_t nseg = ntile * CT_PARTS;
    const int64_t len = (nseg + 31) / 32;
    const int64_t s0 = min((int64_t)lane * len, nseg), s1 = min(s0 + len, nseg);
    double z = 0.0, w = 1.0, Qe = 0.0, Se = 0.0, Qs = 0.0, Ss = 0.0, Ex = 0.0;
    for (int64_t sg = s0; sg < s1; ++sg) {
        const int64_t tile = sg / CT_PARTS, part = sg % CT_PARTS;
        const int64_t o = (part * n + i) * ntile + tile;
        const double P1 = part_tau[o], P2 = part_tau[pl + o], Ze = part_tau[2 * pl + o];
        const double P3 = part_tau[3 * pl + o], P4 = part_tau[4 * pl + o], X = part_tau[5 * pl + o];
        const double Ae = part_tau[6 * pl + o];
        Qe = fma(w, P1, Qe);
        Se += fma(z, P1, P2);
        Qs = fma(w, P3, Qs);
        Ss += fma(z, P3, P4);
        Ex += X;
        z = fma(Ae, z, Ze);
        w *= Ae;
    }
    double v = z, m = w;
    for (int d = 1; d < 32; d <<= 1) {
        const double o = __shfl_up_sync(0xffffffffu, v, d), om = __shfl_up_sync(0xffffffffu, m, d);
        if (lane >= d) {
            v = fma(m, o, v);
            m *= om;
        }
    }
    double zin = __shfl_up_sync(0xffffffffu, v, 1);
    if (lane == 0) zin = 0.0;
    double integ = fma(zin, Qe, Se);
    double spk = fma(zin, Qs, Ss);
    integ = warp_sum(integ);
    spk = warp_sum(spk);
    Ex = warp_sum(Ex);
    if (lane == 0) rows[i] = spk / (tau * tau) - eb[i] * (integ / tau + Ex);
}

cudaError_t launch_tau_rows(glm_ctx* c, double* rows) {
    const Problem& P = c->pb;
    if (P.ct) {
        ct_tau_rows_kernel<<<(P.n + 7) / 8, 256, 0, c->stream>>>(P.n, P.Tpad / tc_tile_t(), P.tau, c->buf.eb,
                                                                 c->buf.part_tau, rows);
        return cudaGetLastError();
    }
    const double A256 = std::exp(-(double)SEG * P.dt / P.tau);
    tau_rows_kernel<<<(P.n + 7) / 8, 256, 0, c->stream>>>(P.n, P.Tpad / tc_tile_t(), P.dt, A256, c->buf.eb,
                                                          c->buf.part_tau, rows);
    return cudaGetLastError();
}

cudaError_t launch_reduce(glm_ctx* c, const float* W, const float* b, double* L_rows, double* G, double* gb,
                          bool want_grad, int64_t ntile, int nsplit, const double* Gacc) {
    const Problem& P = c->pb;
    ReduceArgs A;
    A.n = P.n;
    A.ntile = ntile;
    A.dt = P.dt_int;
    A.W = W;
    A.b = b;
    A.C = c->buf.C;
    A.part_s = c->buf.part_s;
    A.qd = c->buf.qd;
    A.part_e = c->buf.part_e;
    A.planes = P.ct ? CT_PARTS : 1;
    A.r0 = c->row_r0;
    A.r1 = c->row_r1 < 0 ? P.n : c->row_r1;
    A.spk_from_c = P.prec == GLM_PREC_F32 && !P.ct;
    A.part_self = P.self_shift > 0 ? c->buf.part_self : nullptr;
    A.gself = c->buf.gself;
    A.L_rows = L_rows;
    A.gb = gb;
    reduce_rows_kernel<<<(P.n + 7) / 8, 256, 0, c->stream>>>(A);
    if (want_grad && G) {
        const int64_t nn = (int64_t)P.n * P.n;
        const int64_t threads = (nn + SPLIT_EPT - 1) / SPLIT_EPT;
        reduce_grad_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, c->stream>>>(
            nn, nsplit, A.C, c->buf.part_g, Gacc, G, (int64_t)A.r0 * P.n, (int64_t)A.r1 * P.n, P.n, A.part_self ? A.gself : nullptr);
    }
    return cudaGetLastError();
}

cudaError_t launch_total(glm_ctx* c, const double* L_rows, double* out1) {
    total_kernel<<<1, 1024, 0, c->stream>>>(c->pb.n, L_rows, out1);
    return cudaGetLastError();
}

}  // namespace glm
