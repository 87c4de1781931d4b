// Step a2: the spike term of the gradient and of the log-likelihood,
//   C_ij = sum_{t : S_i[t] = 1} X_j[t]   (the sum over v_ij(t_ik) in Eq. 12),
// which does not depend on W or b and is computed once per problem (Sec. 2.3.3, 2.6.1).  With it
//   sum_t S_i[t] U_i[t] = q_i b_i + sum_j W_ij C_ij    and    dL_i/dW_ij = C_ij - dt sum_t e^{U_i[t]} X_j[t].
//
// Block = (16 presynaptic rows j, a part of the time axis, a slice of 1024 postsynaptic rows i), 16 warps,
// two rows i per thread.  For each 1024-bin sub-chunk:
//   staging  every thread starts asynchronous copies (cp.async) of its rows' spike bins in the sub-chunk
//            (up to 24 per row) into shared memory, laid out [spike][row slot][thread] so that the later
//            reads of a warp are conflict-free;
//   phase A  meanwhile the warps scan X_j for the 16 rows into shared memory (warp = one 256-bin segment x
//            4 rows, started from the segment carries);
//   phase B  every thread walks the staged spikes of its rows and accumulates X_j[t] for the 16 rows (spikes
//            beyond the staged 24 are read from global memory).
// X is scanned in double-float (seg_scan_df) and kept in shared memory as hi + lo pairs; every spike's pair
// enters the row's double-float sum (TwoSum on the hi parts, the lo parts added alongside), ~44 significant
// bits in a fixed order: C is exact to far below the FP32 rounding of X, which the log-likelihood of the
// plain FP32 form needs (its spike part is sum_j W_ij C_ij).
#include <cmath>

#include "glm_internal.h"
#include "scan_dev.cuh"

namespace glm {

constexpr int ST_THREADS = 512;
constexpr int ST_JB = 16;                     // presynaptic rows per block
constexpr int ST_SUBSEGS = 4;                 // 1024 bins per sub-chunk
constexpr int ST_SUB = ST_SUBSEGS * SEG;
constexpr int ST_KI = 2;                      // postsynaptic rows per thread
constexpr int ST_ROWS_PER_SLICE = ST_THREADS * ST_KI;
constexpr int ST_CAP = 20;                    // spike bins per row and sub-chunk staged in shared memory
static_assert(ST_THREADS / 32 == ST_SUBSEGS * (ST_JB / 4), "phase A: one warp per (segment, 4 rows)");

// Xs layout: [bin][16 hi floats, 16 lo floats] = 8 chunks of 16 bytes per bin, plus one 16-byte pad after
// every 8 bins; the phase-B loads of one bin are 8 consecutive chunks (one base, immediate offsets).
constexpr int XS_CHUNKS = ST_SUB * 8 + ST_SUB / 8;
constexpr size_t ST_SMEM = (size_t)XS_CHUNKS * 16 + (size_t)ST_CAP * ST_KI * ST_THREADS * 4;
static_assert(ST_SMEM <= 227 * 1024, "shared memory of one block");
__device__ __forceinline__ int xs_base(int bin) { return bin * 8 + (bin >> 3); }

__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ void two_sum(float& hi, float& lo, float x) {
    const float s = hi + x;
    const float bp = s - hi;
    const float e = (hi - (s - bp)) + (x - bp);
    hi = s;
    lo += e;
}

// seg_bits (scan_dev.cuh) with the first 32-spike window already loaded into `sv`
__device__ __forceinline__ uint32_t seg_bits_pre(const int32_t* __restrict__ bins, int64_t cur, int64_t end,
                                                 int64_t t0, int lane, int64_t sv) {
    uint32_t my = 0;
    int64_t s = sv;
    while (true) {
        const bool in = s < t0 + SEG;
        const uint32_t bal = __ballot_sync(FULL, in);
        uint32_t m = bal;
        while (m) {
            const int src = __ffs(m) - 1;
            m &= m - 1;
            const int off = (int)(__shfl_sync(FULL, s, src) - t0);
            if ((off >> 3) == lane) my |= 1u << (off & 7);
        }
        const int c = __popc(bal);
        cur += c;
        if (c < 32) break;
        const int64_t k = cur + lane;
        s = (k < end) ? (int64_t)__ldg(bins + k) : INT64_MAX;
    }
    return my;
}

struct SpikeTermArgs {
    int32_t n;
    int64_t nseg;
    int64_t segs_per_part;
    const int64_t* offs;
    const int32_t* bins;
    const float2* seg_carry;  // double-float pairs
    const int32_t* seg_first;
    // the source trains scanned into X (the spikes, or the spikes shifted by a source delay)
    const int64_t* aoffs;
    const int32_t* abins;
    const int32_t* aseg_first;
    double* C_part;  // [parts][n][n]
};

__global__ void __launch_bounds__(ST_THREADS, 1) spike_term_kernel(const __grid_constant__ ScanConsts K,
                                                                   const __grid_constant__ SpikeTermArgs A) {
    extern __shared__ float4 Xs[];  // [XS_CHUNKS], then the staged spike bins
    int32_t* Sp = reinterpret_cast<int32_t*>(Xs + XS_CHUNKS);  // [ST_CAP][ST_KI][ST_THREADS], bin - sub-chunk start
    const uint32_t sp_addr = (uint32_t)__cvta_generic_to_shared(Sp);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int32_t j0 = blockIdx.x * ST_JB;
    const int64_t part = blockIdx.y;
    const int32_t i_base = blockIdx.z * ST_ROWS_PER_SLICE;
    const float2 pl = make_float2(K.pl_hi[lane], K.pl_lo[lane]);
    const int64_t sp0 = part * A.segs_per_part;
    const int64_t sp1 = min(sp0 + A.segs_per_part, A.nseg);
    const int seg_w = warp & (ST_SUBSEGS - 1);   // phase A: this warp's segment
    const int grp_w = warp / ST_SUBSEGS;         // and its 4 of the 16 presynaptic rows

    float acc_hi[ST_KI][ST_JB], acc_lo[ST_KI][ST_JB];
    int64_t cur[ST_KI], rend[ST_KI], nxt[ST_KI];
#pragma unroll
    for (int k = 0; k < ST_KI; ++k) {
#pragma unroll
        for (int jj = 0; jj < ST_JB; ++jj) acc_hi[k][jj] = acc_lo[k][jj] = 0.f;
        const int32_t i = i_base + threadIdx.x + k * ST_THREADS;
        cur[k] = rend[k] = nxt[k] = 0;
        if (i < A.n && sp0 < sp1) {
            const int64_t o0 = A.offs[i];
            cur[k] = o0 + A.seg_first[(int64_t)i * A.nseg + sp0];
            rend[k] = A.offs[i + 1];
            const int64_t sn = min(sp1, sp0 + ST_SUBSEGS);
            nxt[k] = (sn < A.nseg) ? o0 + A.seg_first[(int64_t)i * A.nseg + sn] : rend[k];
        }
    }

    for (int64_t sc = sp0; sc < sp1; sc += ST_SUBSEGS) {
        const int64_t tb = sc * SEG;
        // ---- staging: this sub-chunk's spike bins of the thread's rows, asynchronously ----
        int64_t k1[ST_KI];
        int cnt[ST_KI];
#pragma unroll
        for (int k = 0; k < ST_KI; ++k) {
            k1[k] = nxt[k];
            cnt[k] = (int)(k1[k] - cur[k]);
            const int c = min(cnt[k], ST_CAP);
            for (int u = 0; u < c; ++u)
                cp_async4(sp_addr + 4u * (uint32_t)((u * ST_KI + k) * ST_THREADS + threadIdx.x), A.bins + cur[k] + u);
        }
        cp_async_commit();
        // end of each row's spikes in the next sub-chunk, for the next staging step
        const int64_t s2 = min(sp1, sc + 2 * ST_SUBSEGS);
#pragma unroll
        for (int k = 0; k < ST_KI; ++k) {
            const int32_t i = i_base + threadIdx.x + k * ST_THREADS;
            if (i < A.n && sc + ST_SUBSEGS < sp1)
                nxt[k] = (s2 < A.nseg) ? A.offs[i] + A.seg_first[(int64_t)i * A.nseg + s2] : rend[k];
        }
        // ---- phase A: X_j for the 16 rows over this sub-chunk, into shared memory ----
        const int64_t s = sc + seg_w;
        if (s < sp1) {
            const int64_t t0 = s * SEG;
            float2 xs[4];
            int64_t rc[4], re[4], sv[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int32_t r = j0 + grp_w * 4 + k;
                xs[k] = make_float2(0.f, 0.f);
                rc[k] = re[k] = 0;
                if (r < A.n) {
                    xs[k] = A.seg_carry[(int64_t)r * A.nseg + s];
                    rc[k] = A.aoffs[r] + A.aseg_first[(int64_t)r * A.nseg + s];
                    re[k] = A.aoffs[r + 1];
                }
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int64_t kk = rc[k] + lane;
                sv[k] = (kk < re[k]) ? (int64_t)__ldg(A.abins + kk) : INT64_MAX;
            }
            float* xf = reinterpret_cast<float*>(Xs);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t bits = seg_bits_pre(A.abins, rc[k], re[k], t0, lane, sv[k]);
                float2 v[8];
                seg_scan_df(K, xs[k], bits, pl, lane, v);
#pragma unroll
                for (int m = 0; m < 8; ++m) {
                    const int bin = seg_w * SEG + 8 * lane + m;
                    xf[4 * xs_base(bin) + grp_w * 4 + k] = v[m].x;
                    xf[4 * xs_base(bin) + 16 + grp_w * 4 + k] = v[m].y;
                }
            }
        }
        cp_async_wait_all();
        __syncthreads();
        // ---- phase B: the spikes of this thread's postsynaptic rows in the sub-chunk ----
        auto add_bin = [&](int k, int t) {
            const float4* xp = Xs + xs_base(t);
#pragma unroll
            for (int ch = 0; ch < 4; ++ch) {
                const float4 h = xp[ch], l = xp[4 + ch];
                two_sum(acc_hi[k][4 * ch + 0], acc_lo[k][4 * ch + 0], h.x);
                two_sum(acc_hi[k][4 * ch + 1], acc_lo[k][4 * ch + 1], h.y);
                two_sum(acc_hi[k][4 * ch + 2], acc_lo[k][4 * ch + 2], h.z);
                two_sum(acc_hi[k][4 * ch + 3], acc_lo[k][4 * ch + 3], h.w);
                acc_lo[k][4 * ch + 0] += l.x;
                acc_lo[k][4 * ch + 1] += l.y;
                acc_lo[k][4 * ch + 2] += l.z;
                acc_lo[k][4 * ch + 3] += l.w;
            }
        };
#pragma unroll
        for (int k = 0; k < ST_KI; ++k) {
            const int c = min(cnt[k], ST_CAP);
            const int32_t* sk = Sp + k * ST_THREADS + threadIdx.x;
#pragma unroll 2
            for (int u = 0; u < c; ++u) add_bin(k, sk[u * ST_KI * ST_THREADS] - (int)tb);
            for (int u = ST_CAP; u < cnt[k]; ++u)  // beyond the staged spikes (rows firing fast)
                add_bin(k, (int)(__ldg(A.bins + cur[k] + u) - tb));
            cur[k] = k1[k];
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

// Parts of the time axis: enough blocks for about three full waves of one block per SM.
int spike_term_parts(const glm_ctx* c) {
    const int64_t nsub = (c->pb.nseg + ST_SUBSEGS - 1) / ST_SUBSEGS;
    const int64_t groups = (c->pb.n + ST_JB - 1) / ST_JB;
    const int64_t slices = (c->pb.n + ST_ROWS_PER_SLICE - 1) / ST_ROWS_PER_SLICE;
    int64_t p = (3 * (int64_t)c->sm_count + groups * slices - 1) / (groups * slices);
    if (p < 1) p = 1;
    if (p > nsub) p = nsub;
    if (p > 64) p = 64;
    return (int)p;
}

cudaError_t launch_spike_term(glm_ctx* c, double* out) {
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
    A.aoffs = c->buf.aoffs;
    A.abins = c->buf.abins;
    A.aseg_first = c->buf.aseg_first;
    A.C_part = c->buf.C_part;
    const size_t smem = ST_SMEM;
    dim3 grid((P.n + ST_JB - 1) / ST_JB, parts, (P.n + ST_ROWS_PER_SLICE - 1) / ST_ROWS_PER_SLICE);
    cudaError_t e = cudaFuncSetAttribute(spike_term_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    spike_term_kernel<<<grid, ST_THREADS, smem, c->stream>>>(c->sc, A);
    const int64_t nn = (int64_t)P.n * P.n;
    spike_term_reduce_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, c->stream>>>(nn, parts, c->buf.C_part, out);
    return cudaGetLastError();
}

}  // namespace glm
