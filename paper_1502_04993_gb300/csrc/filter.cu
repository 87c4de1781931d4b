// Step a0/a1: spike ingest and the filter scan X_j[t] = a X_j[t-1] + S_j[t-1] (Eq. 13 on the grid; the
// exponential kernel h(t) = H(t) exp(-t/tau) of Sec. 2.2 with a one-bin delay).
//
//   carry pass  (double-float, O(q + n * nseg)):  per row and 256-bin segment, X at the segment start and the
//               index of the first spike in or after the segment.
//   write pass  (FP32 scan for the 16-bit forms, writing at ~80 % of the copy bandwidth, bound by
//               instruction issue; double-float scan for the FP32 form):  the segments of a 4096-bin chunk
//               are scanned in order, starting from the carry, and stored as
//                 F32:    X row-major [n][Tpad]
//                 16-bit: X_hi and X_lo = X - X_hi rounded once more, both bin-blocked [Tpad / 64][n][64],
//                         the layout both tensor-core products read (and, on the grid, the spike raster)
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cmath>

#include "glm_internal.h"
#include "scan_dev.cuh"

namespace glm {

void fill_scan_consts(double a, ScanConsts* sc) {
    auto split = [](double v, float* hi, float* lo) {
        const float h = (float)v;
        *hi = h;
        *lo = (float)(v - (double)h);
    };
    split(a, &sc->a_hi, &sc->a_lo);
    for (int m = 0; m <= 8; ++m) split(std::pow(a, (double)m), &sc->pm_hi[m], &sc->pm_lo[m]);
    for (int d = 0; d < 5; ++d) split(std::pow(a, 8.0 * (1 << d)), &sc->ps_hi[d], &sc->ps_lo[d]);
    for (int l = 0; l < 32; ++l) split(std::pow(a, 8.0 * l), &sc->pl_hi[l], &sc->pl_lo[l]);
}

// Segment-first indices and, in seg_local (when given), the contribution of each segment's own spikes to X
// at the next segment start: sum_{t in seg s} a^(256 (s+1) - 1 - t) on the grid; with continuous-time
// columns (ctime given) sum exp(-(c_end - c_{t+1}) / tau), a source t arriving at column t+1.
// Block per row, SL_W warps; warp w owns a contiguous range of segments and finds its spikes by a search in
// the row's sorted bins.  It walks them 32 at a time (the loads of four such steps issued together): the spikes of one
// segment are adjacent lanes, their terms are summed by a shuffle tree over the run, and a run that goes on
// past the 32 lanes is carried to the next step (its partial sum first).  The sums are double-float pairs
// (on the grid the powers a^k come from a shared table of pairs), and the order of the additions depends
// only on the data: the result is reproducible.
constexpr int SL_W = 8;

// First k in [lo0, q) with b[k] >= x (q if none) in the sorted bins of a row, found by the whole warp: each
// round probes 32 points that split the interval in 33 parts, so a row of 10^4 spikes takes 4 dependent
// loads.  Every probe lies inside [lo, hi) and the interval shrinks every round.
__device__ __forceinline__ int64_t warp_lower_bound(const int32_t* __restrict__ b, int64_t lo0, int64_t q, int64_t x,
                                                    int lane) {
    int64_t lo = lo0, hi = q;  // b[k] < x for k < lo, b[k] >= x for hi <= k < q
    while (hi - lo > 32) {
        const int64_t p = lo + (hi - lo) * (lane + 1) / 33;
        const uint32_t below = __ballot_sync(FULL, (int64_t)__ldg(b + p) < x);
        const int c = __popc(below);  // the lanes below x are a prefix
        const int64_t plo = __shfl_sync(FULL, p, c > 0 ? c - 1 : 0);
        const int64_t phi = __shfl_sync(FULL, p, c < 32 ? c : 31);
        if (c > 0) lo = plo + 1;
        if (c < 32) hi = phi;
    }
    const int64_t p = lo + lane;
    return lo + __popc(__ballot_sync(FULL, p < hi && (int64_t)__ldg(b + p) < x));
}

__global__ void __launch_bounds__(SL_W * 32) seg_local_kernel(int32_t n, int64_t nseg, const int64_t* __restrict__ offs,
                                 const int32_t* __restrict__ bins, const double* __restrict__ pow_seg,
                                 const double* __restrict__ ctime, double inv_tau, float2* __restrict__ seg_local,
                                 int32_t* __restrict__ seg_first) {
    __shared__ float2 pw[SEG];
    const int32_t j = blockIdx.x;
    if (j >= n) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t o0 = offs[j], q = offs[j + 1] - o0;
    const int32_t* b = bins + o0;
    float2* loc = seg_local ? seg_local + (int64_t)j * nseg : nullptr;
    int32_t* first = seg_first + (int64_t)j * nseg;
    if (pow_seg)
        for (int k = threadIdx.x; k < SEG; k += blockDim.x) pw[k] = df_from(pow_seg[k]);
    __syncthreads();
    const int64_t sb = nseg * warp / SL_W, se = nseg * (warp + 1) / SL_W;
    if (sb >= se) return;
    if (loc)
        for (int64_t s = sb + lane; s < se; s += 32) loc[s] = make_float2(0.f, 0.f);
    const int64_t k_lo = warp_lower_bound(b, 0, q, sb * SEG, lane);
    const int64_t k_hi = warp_lower_bound(b, k_lo, q, se * SEG, lane);
    __syncwarp();
    int64_t last_s = sb - 1;   // segment of the previous spike of the range
    int64_t open_s = -1;       // segment of the run still open at the end of the previous step
    float2 open_acc = make_float2(0.f, 0.f);  // its partial sum
    for (int64_t base0 = k_lo; base0 < k_hi; base0 += 4 * 32) {
        int32_t pre[4];  // the bins of four steps, loaded together
#pragma unroll
        for (int u = 0; u < 4; ++u) pre[u] = (base0 + 32 * u + lane < k_hi) ? __ldg(b + base0 + 32 * u + lane) : 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t base = base0 + 32 * u;
            if (base >= k_hi) break;
            const int64_t k = base + lane;
            const bool valid = k < k_hi;
            const int64_t bk = valid ? (int64_t)pre[u] : 0;
            const int64_t s = valid ? bk / SEG : INT64_MAX;
            int64_t prev_s = __shfl_up_sync(FULL, s, 1);
            if (lane == 0) prev_s = last_s;
            const bool head = valid && s != prev_s;
            if (head)
                for (int64_t ss = prev_s + 1; ss <= s; ++ss) first[ss] = (int32_t)k;
            const int last_lane = (k_hi - 1 - base < 31) ? (int)(k_hi - 1 - base) : 31;
            if (loc) {
                const int64_t end = valid ? (s + 1) * SEG : 0;
                float2 v = make_float2(0.f, 0.f);
                if (valid) v = ctime ? df_from(exp(-(ctime[end] - ctime[bk + 1]) * inv_tau)) : pw[end - 1 - bk];
                const int32_t s32 = valid ? (int32_t)s : -1;  // segment index (< 2^23) for the shuffles
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {  // lane l: sum over [l, min(l + 2 off, end of its run))
                    const float2 t = make_float2(__shfl_down_sync(FULL, v.x, off), __shfl_down_sync(FULL, v.y, off));
                    const int32_t ts = __shfl_down_sync(FULL, s32, off);
                    if (lane + off < 32 && ts == s32) v = df_add(v, t);
                }
                const bool lead = head || (lane == 0 && valid);  // first lane of a run in this step
                if (lane == 0 && valid && s == open_s) v = df_add(open_acc, v);
                if (lead) loc[s] = v;  // a run carried on to the next step is written again there
                const uint32_t leads = __ballot_sync(FULL, lead) & (0xffffffffu >> (31 - last_lane));
                const int hl = 31 - __clz(leads);
                open_acc = make_float2(__shfl_sync(FULL, v.x, hl), __shfl_sync(FULL, v.y, hl));
                open_s = __shfl_sync(FULL, s, hl);
            }
            last_s = __shfl_sync(FULL, s, last_lane);
        }
    }
    for (int64_t ss = last_s + 1 + lane; ss < se; ss += 32) first[ss] = (int32_t)k_hi;
}

// Block per row, in place: seg_carry[s] <- X_j[256 s], with X_j[256 (s+1)] = A_s X_j[256 s] + local[s]
// (A_s = a^256, or mul_seg[s] for continuous-time columns).  The row goes through shared memory in chunks of
// CS segments, read and written with coalesced accesses: each thread composes the affine maps of its 8
// consecutive segments (multiplier M, offset V), a block scan over the threads composes them in order,
// and each thread then rewrites its segments from its carry-in.  The chunk's carry-out starts the next
// chunk.  All values are double-float pairs (~44 bits; the readers round the carries to FP32); the order of
// the operations is fixed: the result is reproducible.
constexpr int SC_T = 256, SC_E = 8, SC_CS = SC_T * SC_E;

__device__ __forceinline__ int sc_pad(int k) { return k + (k >> 3); }  // one pad per 8 pairs: no bank conflicts

__device__ __forceinline__ float2 shfl_up_f2(float2 v, int d) {
    return make_float2(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d));
}

__global__ void __launch_bounds__(SC_T) seg_carry_kernel(int32_t n, int64_t nseg, double a_seg,
                                                         const double* __restrict__ mul_seg, float2* __restrict__ seg) {
    __shared__ float2 sl[SC_CS + SC_CS / 8], sa[SC_CS + SC_CS / 8];
    __shared__ float2 wm[SC_T / 32], wv[SC_T / 32];
    __shared__ float2 s_cin;
    const int32_t j = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (j >= n) return;
    float2* p = seg + (int64_t)j * nseg;
    const float2 a2 = df_from(a_seg), one = make_float2(1.f, 0.f), zero = make_float2(0.f, 0.f);
    if (tid == 0) s_cin = zero;
    for (int64_t c0 = 0; c0 < nseg; c0 += SC_CS) {
        const int len = (int)min((int64_t)SC_CS, nseg - c0);
        __syncthreads();  // s_cin of the previous chunk is written; the buffers are free
        for (int k = tid; k < SC_CS; k += SC_T) {
            sl[sc_pad(k)] = k < len ? p[c0 + k] : zero;
            sa[sc_pad(k)] = k < len ? (mul_seg ? df_from(mul_seg[c0 + k]) : a2) : one;
        }
        __syncthreads();
        // this thread's map over segments [tid E, tid E + E)
        float2 M = one, V = zero;
#pragma unroll
        for (int e = 0; e < SC_E; ++e) {
            const int k = sc_pad(tid * SC_E + e);
            V = df_fma(sa[k], V, sl[k]);
            M = df_mul(M, sa[k]);
        }
        // inclusive scan of the maps over the threads: (M, V) after (M', V') is (M M', M V' + V)
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const float2 oM = shfl_up_f2(M, d), oV = shfl_up_f2(V, d);
            if (lane >= d) {
                V = df_fma(M, oV, V);
                M = df_mul(M, oM);
            }
        }
        if (lane == 31) {
            wm[wid] = M;
            wv[wid] = V;
        }
        __syncthreads();
        // carry into this thread's first segment: chunk carry-in through the earlier warps, then the
        // earlier lanes of this warp
        float2 cin = s_cin;
        for (int w = 0; w < wid; ++w) cin = df_fma(wm[w], cin, wv[w]);
        {
            const float2 pM = shfl_up_f2(M, 1), pV = shfl_up_f2(V, 1);
            if (lane > 0) cin = df_fma(pM, cin, pV);
        }
#pragma unroll
        for (int e = 0; e < SC_E; ++e) {
            const int k = sc_pad(tid * SC_E + e);
            const float2 l = sl[k];
            sl[k] = cin;
            cin = df_fma(sa[k], cin, l);
        }
        if (tid == SC_T - 1) s_cin = cin;
        __syncthreads();
        for (int k = tid; k < len; k += SC_T) p[c0 + k] = sl[sc_pad(k)];
    }
}

constexpr int CHUNK_SEGS = 16;  // 4096 bins per warp unit: X is chained in FP32 within a unit and restarted
                                // from the segment carry at every unit start (chunks of X start on unit bounds)
constexpr int FW_WARPS = 4;
constexpr int FW16_RPW = 4;  // rows per warp of the 16-bit filter

template <typename T16>
__device__ __forceinline__ uint32_t pack2(float lo, float hi);
template <>
__device__ __forceinline__ uint32_t pack2<__nv_bfloat16>(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}
template <>
__device__ __forceinline__ uint32_t pack2<__half>(float lo, float hi) {
    __half2 v = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

// X_hi and X_lo words of two adjacent values: one paired conversion each, the hi word kept as converted
// (the same rounding as two separate conversions, in fewer instructions; the filter is issue-bound)
template <typename T16>
__device__ __forceinline__ void split_pair(float a, float b, uint32_t& hi, uint32_t& lo);
template <>
__device__ __forceinline__ void split_pair<__nv_bfloat16>(float a, float b, uint32_t& hi, uint32_t& lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 hf = __bfloat1622float2(h);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = pack2<__nv_bfloat16>(a - hf.x, b - hf.y);
}
template <>
__device__ __forceinline__ void split_pair<__half>(float a, float b, uint32_t& hi, uint32_t& lo) {
    const __half2 h = __floats2half2_rn(a, b);
    const float2 hf = __half22float2(h);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = pack2<__half>(a - hf.x, b - hf.y);
}

struct FilterArgs {
    int32_t n;
    int64_t T, nseg, Tpad, ldn;
    int32_t ngroups;
    int64_t nchunks;
    int64_t s_begin, s_end;  // segments written; the buffers start at bin SEG s_begin
    const int64_t* offs;
    const int32_t* bins;
    const float2* seg_carry;  // [n][nseg] X at each segment start, double-float pairs
    const int32_t* seg_first;
    void* X;
    void* Xlo;  // 16-bit forms: X_lo
    const float* col_a;  // continuous-time columns: decay of each column
    void* S;             // 16-bit filter: also the spike raster (0 / 1), bin-blocked like X, or null
    uint16_t one;        // the 16-bit word of 1
};

// F32 X, one warp per (8 rows, 4096-bin chunk).  The scan runs in double-float and each stored value is
// rounded once from it: the stored X is the correctly rounded X (the plain FP32 form's L needs X free of
// systematic rounding to reach ~1e-9 relative).  The filter runs once per problem, so the extra arithmetic
// does not recur in the fit.
__global__ void __launch_bounds__(FW_WARPS * 32) filter_cache_f32_kernel(const __grid_constant__ ScanConsts K,
                                                                         const __grid_constant__ FilterArgs A) {
    const int lane = threadIdx.x & 31;
    const int64_t wg = (int64_t)blockIdx.x * FW_WARPS + (threadIdx.x >> 5);
    const int64_t c = wg / A.ngroups;
    const int32_t g = (int32_t)(wg % A.ngroups);
    if (c >= A.nchunks) return;
    const float2 pl = make_float2(K.pl_hi[lane], K.pl_lo[lane]);
    const int64_t s0 = A.s_begin + c * CHUNK_SEGS;
    const int64_t s1 = min(s0 + (int64_t)CHUNK_SEGS, A.s_end);
    for (int k = 0; k < 8; ++k) {
        const int32_t r = g * 8 + k;
        if (r >= A.n) break;
        float2 xs = A.seg_carry[(int64_t)r * A.nseg + s0];
        int64_t cur = A.offs[r] + A.seg_first[(int64_t)r * A.nseg + s0];
        const int64_t end = A.offs[r + 1];
        for (int64_t s = s0; s < s1; ++s) {
            const int64_t t0 = s * SEG;
            const uint32_t bits = seg_bits(A.bins, cur, end, t0, lane);
            float2 v[8];
            xs = seg_scan_df(K, xs, bits, pl, lane, v);
            float4* dst = reinterpret_cast<float4*>(reinterpret_cast<float*>(A.X) + (int64_t)r * A.Tpad + t0 + 8 * lane);
            dst[0] = make_float4(df_f(v[0]), df_f(v[1]), df_f(v[2]), df_f(v[3]));
            dst[1] = make_float4(df_f(v[4]), df_f(v[5]), df_f(v[6]), df_f(v[7]));
        }
    }
}

// 16-bit caches: X_hi and X_lo, X_lo = X - X_hi rounded again, both bin-blocked [Tpad / 64][n][64] (bins
// [64 b, 64 b + 64) of row r at (b n + r) 64), the layout the tensor-core products read; X_hi alone (the
// round-to-nearest 16-bit X) when A.Xlo is null (XLO false).  One warp per (RPW rows, 4096-bin chunk): each lane stores
// its 8 bins of a row as one 16-byte word of X_hi and one of X_lo, so every warp store covers four whole
// 128-byte lines.
template <typename T16, int RPW, bool XLO>
__global__ void __launch_bounds__(FW_WARPS * 32) filter_cache16_kernel(const __grid_constant__ ScanConsts K,
                                                                       const __grid_constant__ FilterArgs A) {
    const int lane = threadIdx.x & 31;
    const int64_t wg = (int64_t)blockIdx.x * FW_WARPS + (threadIdx.x >> 5);
    const int64_t c = wg / A.ngroups;
    const int32_t g = (int32_t)(wg % A.ngroups);
    if (c >= A.nchunks) return;
    const float pl_hi = K.pl_hi[lane], pl_lo = K.pl_lo[lane];
    const int64_t s0 = A.s_begin + c * CHUNK_SEGS;
    const int64_t s1 = min(s0 + (int64_t)CHUNK_SEGS, A.s_end);
    float xs[RPW];
    int64_t cur[RPW], end[RPW];
#pragma unroll
    for (int k = 0; k < RPW; ++k) {
        const int32_t r = g * RPW + k;
        if (r < A.n) {
            xs[k] = df_f(A.seg_carry[(int64_t)r * A.nseg + s0]);
            cur[k] = A.offs[r] + A.seg_first[(int64_t)r * A.nseg + s0];
            end[k] = A.offs[r + 1];
        } else {
            xs[k] = 0.f;
            cur[k] = 0;
            end[k] = 0;
        }
    }
    T16* Xh = reinterpret_cast<T16*>(A.X);
    T16* Xl = reinterpret_cast<T16*>(A.Xlo);
    for (int64_t s = s0; s < s1; ++s) {
        const int64_t t0 = s * SEG;
        const int64_t tl = t0 + 8 * lane;
#pragma unroll
        for (int k = 0; k < RPW; ++k) {
            const int32_t r = g * RPW + k;
            const uint32_t bits = seg_bits(A.bins, cur[k], end[k], t0, lane);
            float v[8];
            xs[k] = seg_scan16(K, xs[k], bits, pl_hi, pl_lo, lane, v);
            uint32_t ph[4], pl[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                if (XLO) split_pair<T16>(v[2 * p], v[2 * p + 1], ph[p], pl[p]);
                else ph[p] = pack2<T16>(v[2 * p], v[2 * p + 1]);
            }
            if (r < A.n) {
                const int64_t tb = tl - A.s_begin * SEG;  // bin within the buffers
                const int64_t o = ((tb >> 6) * A.n + r) * 64 + (tb & 63);
                *reinterpret_cast<uint4*>(Xh + o) = make_uint4(ph[0], ph[1], ph[2], ph[3]);
                if (XLO) *reinterpret_cast<uint4*>(Xl + o) = make_uint4(pl[0], pl[1], pl[2], pl[3]);
                if (A.S) {  // the sources are the rows' own spikes: bits is also row r's raster here
                    uint32_t sw[4];
#pragma unroll
                    for (int p = 0; p < 4; ++p)
                        sw[p] = (((bits >> (2 * p)) & 1u) ? (uint32_t)A.one : 0u) |
                                (((bits >> (2 * p + 1)) & 1u) ? ((uint32_t)A.one << 16) : 0u);
                    *reinterpret_cast<uint4*>(reinterpret_cast<uint16_t*>(A.S) + o) = make_uint4(sw[0], sw[1], sw[2], sw[3]);
                }
            }
        }
    }
}

// Continuous-time columns: as filter_cache16_kernel with the decay of each column (seg_scan_ct); the
// multipliers of a segment are formed once for the 8 rows of the warp.
template <typename T16>
__global__ void __launch_bounds__(FW_WARPS * 32) filter_cache16_ct_kernel(const __grid_constant__ FilterArgs A) {
    const int lane = threadIdx.x & 31;
    const int64_t wg = (int64_t)blockIdx.x * FW_WARPS + (threadIdx.x >> 5);
    const int64_t c = wg / A.ngroups;
    const int32_t g = (int32_t)(wg % A.ngroups);
    if (c >= A.nchunks) return;
    const int64_t s0 = A.s_begin + c * CHUNK_SEGS;
    const int64_t s1 = min(s0 + (int64_t)CHUNK_SEGS, A.s_end);
    float xs[8];
    int64_t cur[8], end[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int32_t r = g * 8 + k;
        if (r < A.n) {
            xs[k] = df_f(A.seg_carry[(int64_t)r * A.nseg + s0]);
            cur[k] = A.offs[r] + A.seg_first[(int64_t)r * A.nseg + s0];
            end[k] = A.offs[r + 1];
        } else {
            xs[k] = 0.f;
            cur[k] = 0;
            end[k] = 0;
        }
    }
    T16* Xh = reinterpret_cast<T16*>(A.X);
    T16* Xl = reinterpret_cast<T16*>(A.Xlo);
    for (int64_t s = s0; s < s1; ++s) {
        const int64_t t0 = s * SEG;
        const int64_t tl = t0 + 8 * lane;
        CtSegMul S;
        ct_seg_setup(A.col_a, t0, lane, S);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int32_t r = g * 8 + k;
            const uint32_t bits = seg_bits(A.bins, cur[k], end[k], t0, lane);
            float v[8];
            xs[k] = seg_scan_ct(S, xs[k], bits, lane, v);
            uint32_t ph[4], pl[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) split_pair<T16>(v[2 * p], v[2 * p + 1], ph[p], pl[p]);
            if (r < A.n) {
                const int64_t tb = tl - A.s_begin * SEG;
                const int64_t o = ((tb >> 6) * A.n + r) * 64 + (tb & 63);
                *reinterpret_cast<uint4*>(Xh + o) = make_uint4(ph[0], ph[1], ph[2], ph[3]);
                *reinterpret_cast<uint4*>(Xl + o) = make_uint4(pl[0], pl[1], pl[2], pl[3]);
            }
        }
    }
}

struct RangeArgs {
    int32_t n;
    int64_t T, nseg;
    int32_t ngroups;
    int64_t s_begin, nchunks;
    int64_t t0, t_len, ldx;
    int dtype;
    const int64_t* offs;
    const int32_t* bins;
    const float2* seg_carry;  // [n][nseg] X at each segment start, double-float pairs
    const int32_t* seg_first;
    void* out;
};

// X[:, t0 : t0 + t_len] into a caller buffer (any leading dimension, element-wise stores).
__global__ void __launch_bounds__(FW_WARPS * 32) filter_range_kernel(const __grid_constant__ ScanConsts K,
                                                                     const __grid_constant__ RangeArgs A) {
    const int lane = threadIdx.x & 31;
    const int64_t wg = (int64_t)blockIdx.x * FW_WARPS + (threadIdx.x >> 5);
    const int64_t c = wg / A.ngroups;
    const int32_t g = (int32_t)(wg % A.ngroups);
    if (c >= A.nchunks) return;
    const float2 pl = make_float2(K.pl_hi[lane], K.pl_lo[lane]);
    const int64_t s0 = A.s_begin + c * CHUNK_SEGS;
    const int64_t s1 = min(s0 + (int64_t)CHUNK_SEGS, A.nseg);
    const int64_t te = A.t0 + A.t_len;
    for (int k = 0; k < 8; ++k) {
        const int32_t r = g * 8 + k;
        if (r >= A.n) break;
        float2 xs = A.seg_carry[(int64_t)r * A.nseg + s0];
        int64_t cur = A.offs[r] + A.seg_first[(int64_t)r * A.nseg + s0];
        const int64_t end = A.offs[r + 1];
        for (int64_t s = s0; s < s1; ++s) {
            const int64_t t0 = s * SEG;
            if (t0 >= te) break;
            const uint32_t bits = seg_bits(A.bins, cur, end, t0, lane);
            float2 v[8];
            xs = seg_scan_df(K, xs, bits, pl, lane, v);  // as the FP32 cache: X rounded once
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                const int64_t t = t0 + 8 * lane + m;
                if (t < A.t0 || t >= te) continue;
                const int64_t o = (int64_t)r * A.ldx + (t - A.t0);
                const float x = df_f(v[m]);
                if (A.dtype == GLM_DTYPE_F32)
                    reinterpret_cast<float*>(A.out)[o] = x;
                else if (A.dtype == GLM_DTYPE_BF16)
                    reinterpret_cast<__nv_bfloat16*>(A.out)[o] = __float2bfloat16_rn(x);
                else
                    reinterpret_cast<__half*>(A.out)[o] = __float2half_rn(x);
            }
        }
    }
}

// The spike raster S (1 at every spike, 0 elsewhere) in 16 bits, bin-blocked like X, for the tensor-core
// spike term C = S X^T: one warp per (8 rows, 4096-bin unit), each lane writing its 8 bins of a row as one
// 16-byte word, so every bin of the buffers is written once (no separate clearing pass).
__global__ void __launch_bounds__(FW_WARPS * 32) spike_raster16_kernel(const __grid_constant__ FilterArgs A,
                                                                       uint16_t one) {
    const int lane = threadIdx.x & 31;
    const int64_t wg = (int64_t)blockIdx.x * FW_WARPS + (threadIdx.x >> 5);
    const int64_t c = wg / A.ngroups;
    const int32_t g = (int32_t)(wg % A.ngroups);
    if (c >= A.nchunks) return;
    const int64_t s0 = A.s_begin + c * CHUNK_SEGS;
    const int64_t s1 = min(s0 + (int64_t)CHUNK_SEGS, A.s_end);
    uint16_t* S = reinterpret_cast<uint16_t*>(A.X);
#pragma unroll 1
    for (int k = 0; k < 8; ++k) {
        const int32_t r = g * 8 + k;
        if (r >= A.n) break;
        int64_t cur = A.offs[r] + A.seg_first[(int64_t)r * A.nseg + s0];
        const int64_t end = A.offs[r + 1];
        for (int64_t s = s0; s < s1; ++s) {
            const int64_t t0 = s * SEG;
            const uint32_t bits = seg_bits(A.bins, cur, end, t0, lane);
            uint32_t w[4];
#pragma unroll
            for (int p = 0; p < 4; ++p)
                w[p] = (((bits >> (2 * p)) & 1u) ? (uint32_t)one : 0u) |
                       (((bits >> (2 * p + 1)) & 1u) ? ((uint32_t)one << 16) : 0u);
            const int64_t tb = t0 + 8 * lane - A.s_begin * SEG;  // bin within the buffer
            *reinterpret_cast<uint4*>(S + ((tb >> 6) * A.n + r) * 64 + (tb & 63)) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

cudaError_t launch_spike_raster(glm_ctx* c, void* out, int64_t s_begin, int64_t s_end) {
    const Problem& P = c->pb;
    FilterArgs A;
    A.n = P.n;
    A.T = P.T;
    A.nseg = P.nseg;
    A.Tpad = P.Tpad;
    A.ldn = c->buf.ldn;
    A.ngroups = (P.n + 7) / 8;
    A.s_begin = s_begin;
    A.s_end = s_end;
    A.nchunks = (s_end - s_begin + CHUNK_SEGS - 1) / CHUNK_SEGS;
    A.offs = c->buf.offs;
    A.bins = c->buf.bins;
    A.seg_carry = c->buf.seg_carry;
    A.seg_first = c->buf.seg_first;
    A.X = out;
    A.Xlo = nullptr;
    A.col_a = nullptr;
    A.S = nullptr;
    const uint16_t one = (P.prec == GLM_PREC_BF16) ? 0x3F80u : 0x3C00u;
    const int64_t warps = (int64_t)A.ngroups * A.nchunks;
    spike_raster16_kernel<<<(unsigned)((warps + FW_WARPS - 1) / FW_WARPS), FW_WARPS * 32, 0, c->stream>>>(A, one);
    return cudaGetLastError();
}

// Spike ingest check on the device, for a CSR whose offsets the host has checked (offs[0] = 0, non-decreasing,
// offs[n] = q): every bin inside [0, T) and the bins of each row strictly increasing.  A fault at index k has
// the key 2k (bin out of range) or 2k + 1 (not above the row's previous bin); the smallest key is kept, so the
// host names the same first fault as a pass over the rows in order.  Index k starts a row when some offs[i]
// equals k (binary search; needed only where bins[k] <= bins[k - 1]).
__global__ void __launch_bounds__(256) check_bins_kernel(int32_t n, int64_t q, int64_t T,
                                                         const int64_t* __restrict__ offs,
                                                         const int32_t* __restrict__ bins,
                                                         unsigned long long* __restrict__ first_bad) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < q; k += stride) {
        const int32_t s = __ldg(bins + k);
        unsigned long long key = ~0ull;
        if (s < 0 || (int64_t)s >= T) {
            key = 2ull * (unsigned long long)k;
        } else if (k > 0 && s <= __ldg(bins + k - 1)) {
            int32_t lo = 0, hi = n;  // offs[lo] <= k < offs[hi] is kept; offs[0] = 0 <= k and offs[n] = q > k
            while (hi - lo > 1) {
                const int32_t mid = lo + (hi - lo) / 2;
                if (__ldg(offs + mid) <= k) lo = mid; else hi = mid;
            }
            if (__ldg(offs + lo) != k) key = 2ull * (unsigned long long)k + 1ull;
        }
        if (key != ~0ull) atomicMin(first_bad, key);
    }
}

cudaError_t launch_check_bins(glm_ctx* c, int32_t n, int64_t q, int64_t T, const int64_t* offs, const int32_t* bins,
                              unsigned long long* first_bad) {
    cudaError_t e = cudaMemsetAsync(first_bad, 0xFF, sizeof(unsigned long long), c->stream);
    if (e != cudaSuccess || q <= 0) return e;
    const int64_t blocks = std::min<int64_t>((q + 255) / 256, (int64_t)c->sm_count * 8);
    check_bins_kernel<<<(unsigned)blocks, 256, 0, c->stream>>>(n, q, T, offs, bins, first_bad);
    return cudaGetLastError();
}

cudaError_t launch_carry(glm_ctx* c) {
    const Problem& P = c->pb;
    const Buffers& B = c->buf;
    if (P.ct) {
        // first spike per segment of the spike columns; carries of the arrival sources
        seg_local_kernel<<<P.n, SL_W * 32, 0, c->stream>>>(P.n, P.nseg, B.offs, B.bins, nullptr, nullptr, 0.0, nullptr,
                                                     B.seg_first);
        seg_local_kernel<<<P.n, SL_W * 32, 0, c->stream>>>(P.n, P.nseg, B.aoffs, B.abins, nullptr, B.ctime, 1.0 / P.tau,
                                                     B.seg_carry, B.aseg_first);
        seg_carry_kernel<<<P.n, SC_T, 0, c->stream>>>(P.n, P.nseg, 0.0, B.seg_mul, B.seg_carry);
        return cudaGetLastError();
    }
    if (P.delay_bins > 1) {
        // delayed sources: first spike per segment of the rows' own spikes; carries of the shifted trains
        seg_local_kernel<<<P.n, SL_W * 32, 0, c->stream>>>(P.n, P.nseg, B.offs, B.bins, nullptr, nullptr, 0.0, nullptr,
                                                     B.seg_first);
        seg_local_kernel<<<P.n, SL_W * 32, 0, c->stream>>>(P.n, P.nseg, B.aoffs, B.abins, B.pow_seg, nullptr, 0.0,
                                                     B.seg_carry, B.aseg_first);
    } else {
        seg_local_kernel<<<P.n, SL_W * 32, 0, c->stream>>>(P.n, P.nseg, B.offs, B.bins, B.pow_seg, nullptr, 0.0,
                                                     B.seg_carry, B.seg_first);
    }
    const double a_seg = std::exp(-(double)SEG * P.dt / P.tau);
    seg_carry_kernel<<<P.n, SC_T, 0, c->stream>>>(P.n, P.nseg, a_seg, nullptr, B.seg_carry);
    return cudaGetLastError();
}

cudaError_t launch_filter_cache(glm_ctx* c, int64_t s_begin, int64_t s_end, void* raster) {
    const Problem& P = c->pb;
    FilterArgs A;
    A.n = P.n;
    A.T = P.T;
    A.nseg = P.nseg;
    A.Tpad = P.Tpad;
    A.ldn = c->buf.ldn;
    A.ngroups = (P.n + 7) / 8;
    A.s_begin = s_begin;
    A.s_end = s_end < 0 ? P.nseg : s_end;
    A.nchunks = (A.s_end - A.s_begin + CHUNK_SEGS - 1) / CHUNK_SEGS;
    A.offs = c->buf.aoffs;  // the source trains (the spikes, or the spikes shifted by a delay)
    A.bins = c->buf.abins;
    A.seg_carry = c->buf.seg_carry;
    A.seg_first = c->buf.aseg_first;
    A.X = c->buf.X;
    A.Xlo = c->buf.Xlo;
    A.col_a = c->buf.col_a;
    A.S = raster;
    A.one = (P.prec == GLM_PREC_BF16) ? 0x3F80u : 0x3C00u;
    if (P.ct) {
        A.offs = c->buf.aoffs;
        A.bins = c->buf.abins;
        A.seg_first = c->buf.aseg_first;
        const int64_t warps = (int64_t)A.ngroups * A.nchunks;
        const int64_t blocks = (warps + FW_WARPS - 1) / FW_WARPS;
        if (P.prec == GLM_PREC_BF16)
            filter_cache16_ct_kernel<__nv_bfloat16><<<(unsigned)blocks, FW_WARPS * 32, 0, c->stream>>>(A);
        else
            filter_cache16_ct_kernel<__half><<<(unsigned)blocks, FW_WARPS * 32, 0, c->stream>>>(A);
        return cudaGetLastError();
    }
    if (P.prec == GLM_PREC_F32) {
        const int64_t warps = (int64_t)A.ngroups * A.nchunks;
        const int64_t blocks = (warps + FW_WARPS - 1) / FW_WARPS;
        filter_cache_f32_kernel<<<(unsigned)blocks, FW_WARPS * 32, 0, c->stream>>>(c->sc, A);
    } else {
        // four rows per warp: their independent scans overlap, and 56 registers leave room for enough
        // warps to cover the memory latency (eight rows: 80 registers, 1.84 ms at N = 1000, 1.8 M bins;
        // four: 1.69 ms; two: 1.74 ms; one: 1.70 ms)
        A.ngroups = (P.n + FW16_RPW - 1) / FW16_RPW;
        const int64_t warps = (int64_t)A.ngroups * A.nchunks;
        const int64_t blocks = (warps + FW_WARPS - 1) / FW_WARPS;
        const dim3 g((unsigned)blocks), bl(FW_WARPS * 32);
        if (P.prec == GLM_PREC_BF16) {
            if (A.Xlo) filter_cache16_kernel<__nv_bfloat16, FW16_RPW, true><<<g, bl, 0, c->stream>>>(c->sc, A);
            else filter_cache16_kernel<__nv_bfloat16, FW16_RPW, false><<<g, bl, 0, c->stream>>>(c->sc, A);
        } else {
            if (A.Xlo) filter_cache16_kernel<__half, FW16_RPW, true><<<g, bl, 0, c->stream>>>(c->sc, A);
            else filter_cache16_kernel<__half, FW16_RPW, false><<<g, bl, 0, c->stream>>>(c->sc, A);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_filter_range(glm_ctx* c, int64_t t0, int64_t t_len, void* out, int64_t ldx,
                                glm_dtype_t dtype) {
    const Problem& P = c->pb;
    RangeArgs A;
    A.n = P.n;
    A.T = P.T;
    A.nseg = P.nseg;
    A.ngroups = (P.n + 7) / 8;
    A.s_begin = t0 / SEG;
    const int64_t s_end = (t0 + t_len + SEG - 1) / SEG;
    A.nchunks = (s_end - A.s_begin + CHUNK_SEGS - 1) / CHUNK_SEGS;
    A.t0 = t0;
    A.t_len = t_len;
    A.ldx = ldx;
    A.dtype = (int)dtype;
    A.offs = c->buf.aoffs;
    A.bins = c->buf.abins;
    A.seg_carry = c->buf.seg_carry;
    A.seg_first = c->buf.aseg_first;
    A.out = out;
    const int64_t warps = (int64_t)A.ngroups * A.nchunks;
    const int64_t blocks = (warps + FW_WARPS - 1) / FW_WARPS;
    filter_range_kernel<<<(unsigned)blocks, FW_WARPS * 32, 0, c->stream>>>(c->sc, A);
    return cudaGetLastError();
}

}  // namespace glm
