// Warp-level building blocks of the exponential-recursion scan X[t] = a X[t-1] + S[t-1] (Eq. 13 on
// the time grid).  One warp covers a segment of 256 bins of one row: lane l owns bins
// t0 + 8l .. t0 + 8l + 7.
#pragma once

#include <stdint.h>

#include "glm_internal.h"

namespace glm {

constexpr unsigned FULL = 0xffffffffu;

// Double-float arithmetic: a value is an unevaluated FP32 pair (x = hi, y = lo), ~44-48 significant bits
// (Dekker 1971; Knuth's TwoSum).  The segment carries use it instead of FP64, a scarce pipe on this GPU.
__device__ __forceinline__ float2 df_from(double v) {
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
}
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
    const float s = a.x + b.x;
    const float bp = s - a.x;
    float e = (a.x - (s - bp)) + (b.x - bp);  // a.x + b.x = s + e exactly
    e += a.y + b.y;
    const float h = s + e;
    return make_float2(h, e - (h - s));
}
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
    const float p = a.x * b.x;
    float e = fmaf(a.x, b.x, -p);  // a.x b.x = p + e exactly
    e = fmaf(a.x, b.y, fmaf(a.y, b.x, e));
    const float h = p + e;
    return make_float2(h, e - (h - p));
}
__device__ __forceinline__ float2 df_fma(float2 a, float2 x, float2 y) { return df_add(df_mul(a, x), y); }
// the pair rounded to FP32
__device__ __forceinline__ float df_f(float2 v) { return v.x + v.y; }

// Split product (hi + lo) * x + add in FP32: the multiplier keeps ~48 significant bits.
__device__ __forceinline__ float mul2(float hi, float lo, float x, float add) {
    return fmaf(hi, x, fmaf(lo, x, add));
}

// Spike bits of one row inside the segment [t0, t0 + 256).  `cur` indexes the row's spikes and points
// at the first spike >= t0; it advances past the segment (warp-uniform).  Returns this lane's 8 bits:
// bit m <-> bin t0 + 8 lane + m.
__device__ __forceinline__ uint32_t seg_bits(const int32_t* __restrict__ bins, int64_t& cur, int64_t end,
                                             int64_t t0, int lane) {
    uint32_t my = 0;
    while (true) {
        const int64_t k = cur + lane;
        const int64_t s = (k < end) ? (int64_t)__ldg(bins + k) : INT64_MAX;
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
    }
    return my;
}

// Scan of one segment.  x_seg = X[t0] (all lanes), bits8 = this lane's spike bits, (pl_hi, pl_lo) =
// a^(8 lane).  On return out[m] = X[t0 + 8 lane + m]; the result is X[t0 + 256] (all lanes).
//   local part:   z_m = sum over this lane's spikes j < m of a^(m-1-j)
//   lane start:   X[t_lane] = a^(8 lane) x_seg + sum_{k < lane} a^(8 (lane - 1 - k)) z_8(k)
//                 (Kogge-Stone scan of the affine recurrence with constant multiplier a^8)
//   values:       X[t_lane + m] = a^m X[t_lane] + z_m
// FP32 form of the scan, for the 16-bit caches, whose X_hi + X_lo keep ~17 significant bits: the lane's local
// sums follow the recursion z_{m+1} = a z_m + S_m with a as a hi + lo pair (2 FMAs a bin).  Its FP32 rounding,
// repeated after every spike, biases X by ~0.6 FP32 ulp (~4e-8 relative), far below the 2^-17 of the 16-bit
// pair.  The plain FP32 form uses the double-float scan below (seg_scan_df) and rounds X once.
__device__ __forceinline__ float seg_scan16(const ScanConsts& K, float x_seg, uint32_t bits8, float pl_hi,
                                            float pl_lo, int lane, float out[8]) {
    float z[9];
    z[0] = 0.f;
#pragma unroll
    for (int m = 0; m < 8; ++m) z[m + 1] = mul2(K.a_hi, K.a_lo, z[m], ((bits8 >> m) & 1u) ? 1.f : 0.f);
    float v = z[8];
#pragma unroll
    for (int d = 0; d < 5; ++d) {
        const float o = __shfl_up_sync(FULL, v, 1 << d);
        if (lane >= (1 << d)) v = mul2(K.ps_hi[d], K.ps_lo[d], o, v);
    }
    float ex = __shfl_up_sync(FULL, v, 1);
    if (lane == 0) ex = 0.f;
    const float xl = mul2(pl_hi, pl_lo, x_seg, ex);
#pragma unroll
    for (int m = 0; m < 8; ++m) out[m] = mul2(K.pm_hi[m], K.pm_lo[m], xl, z[m]);
    const float xend = mul2(K.pm_hi[8], K.pm_lo[8], xl, z[8]);
    return __shfl_sync(FULL, xend, 31);
}

__device__ __forceinline__ float2 shfl_up_df(float2 v, int d) {
    return make_float2(__shfl_up_sync(FULL, v.x, d), __shfl_up_sync(FULL, v.y, d));
}

// The scan in double-float arithmetic (~44 significant bits, every multiplier a hi + lo pair): out[m] and
// the result carry X to well below FP32 resolution, so the plain FP32 form rounds each stored value once
// from it (correctly rounded X: no rounding error from the scan itself, whose systematic part, repeated
// after every spike of a train, would otherwise reach ~1e-10 of L).  Same structure as seg_scan16; the
// lane's local sums follow the recursion z_{m+1} = a z_m + S_m, whose double-float roundings are
// ~2^-44 and so negligible.
__device__ __forceinline__ float2 seg_scan_df(const ScanConsts& K, float2 x_seg, uint32_t bits8, float2 pl, int lane,
                                              float2 out[8]) {
    const float2 A = make_float2(K.a_hi, K.a_lo);
    float2 z[9];
    z[0] = make_float2(0.f, 0.f);
#pragma unroll
    for (int m = 0; m < 8; ++m) z[m + 1] = df_add(df_mul(A, z[m]), make_float2((float)((bits8 >> m) & 1u), 0.f));
    float2 v = z[8];
#pragma unroll
    for (int d = 0; d < 5; ++d) {
        const float2 o = shfl_up_df(v, 1 << d);
        if (lane >= (1 << d)) v = df_fma(make_float2(K.ps_hi[d], K.ps_lo[d]), o, v);
    }
    float2 ex = shfl_up_df(v, 1);
    if (lane == 0) ex = make_float2(0.f, 0.f);
    const float2 xl = df_fma(pl, x_seg, ex);
#pragma unroll
    for (int m = 0; m < 8; ++m) out[m] = df_fma(make_float2(K.pm_hi[m], K.pm_lo[m]), xl, z[m]);
    const float2 xend = df_fma(make_float2(K.pm_hi[8], K.pm_lo[8]), xl, z[8]);
    return make_float2(__shfl_sync(FULL, xend.x, 31), __shfl_sync(FULL, xend.y, 31));
}

// Continuous-time columns: the multiplier differs per column, so the powers of a become running products
// of the column decays.  They depend on the columns only and are formed once per segment for all the rows
// a warp scans.  Lane l owns columns t_l = t0 + 8 l .. t_l + 7; al[k] = a_{t_l + k} carries X from column
// t_l + k to t_l + k + 1.
struct CtSegMul {
    float al[8];
    float pk[9];  // pk[k] = al[0] ... al[k-1]
    float ks[5];  // multiplier of this lane's running span at Kogge-Stone step d
    float lp;     // product over all earlier lanes (the a^(8 l) of the constant form)
};

__device__ __forceinline__ void ct_seg_setup(const float* __restrict__ col_a, int64_t t0, int lane, CtSegMul& S) {
    const float4 v0 = __ldg(reinterpret_cast<const float4*>(col_a + t0 + 8 * lane));
    const float4 v1 = __ldg(reinterpret_cast<const float4*>(col_a + t0 + 8 * lane + 4));
    S.al[0] = v0.x;
    S.al[1] = v0.y;
    S.al[2] = v0.z;
    S.al[3] = v0.w;
    S.al[4] = v1.x;
    S.al[5] = v1.y;
    S.al[6] = v1.z;
    S.al[7] = v1.w;
    S.pk[0] = 1.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) S.pk[k + 1] = S.pk[k] * S.al[k];
    float P = S.pk[8];
#pragma unroll
    for (int d = 0; d < 5; ++d) {
        const float o = __shfl_up_sync(FULL, P, 1 << d);
        S.ks[d] = P;
        if (lane >= (1 << d)) P *= o;
    }
    S.lp = __shfl_up_sync(FULL, P, 1);
    if (lane == 0) S.lp = 1.f;
}

// Scan of one segment of columns: as seg_scan16, with the lane's own recursion z_{k+1} = al[k] z_k + S and
// the multipliers of CtSegMul.
__device__ __forceinline__ float seg_scan_ct(const CtSegMul& S, float x_seg, uint32_t bits8, int lane, float out[8]) {
    float z[9];
    z[0] = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) z[k + 1] = fmaf(S.al[k], z[k], (float)((bits8 >> k) & 1u));
    float v = z[8];
#pragma unroll
    for (int d = 0; d < 5; ++d) {
        const float o = __shfl_up_sync(FULL, v, 1 << d);
        if (lane >= (1 << d)) v = fmaf(S.ks[d], o, v);
    }
    float ex = __shfl_up_sync(FULL, v, 1);
    if (lane == 0) ex = 0.f;
    const float xl = fmaf(S.lp, x_seg, ex);
#pragma unroll
    for (int k = 0; k < 8; ++k) out[k] = fmaf(S.pk[k], xl, z[k]);
    return __shfl_sync(FULL, fmaf(S.pk[8], xl, z[8]), 31);
}

}  // namespace glm
