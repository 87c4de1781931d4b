// Warp-level building blocks of the exponential-recursion scan X[t] = a X[t-1] + S[t-1] (Eq. 13 on
// the time grid).  One warp covers a segment of 256 bins of one row: lane l owns bins
// t0 + 8l .. t0 + 8l + 7.
#pragma once

#include <stdint.h>

#include "glm_internal.h"

namespace glm {

constexpr unsigned FULL = 0xffffffffu;

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
//   local part:   z_0 = 0, z_{m+1} = a z_m + S[t_lane + m]   (this lane's own spikes)
//   lane start:   X[t_lane] = a^(8 lane) x_seg + sum_{k < lane} a^(8 (lane - 1 - k)) z_8(k)
//                 (Kogge-Stone scan of the affine recurrence with constant multiplier a^8)
//   values:       X[t_lane + m] = a^m X[t_lane] + z_m
__device__ __forceinline__ float seg_scan(const ScanConsts& K, float x_seg, uint32_t bits8, float pl_hi,
                                          float pl_lo, int lane, float out[8]) {
    float z[8];
    float zz = 0.f;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        z[m] = zz;
        zz = mul2(K.a_hi, K.a_lo, zz, (float)((bits8 >> m) & 1u));
    }
    float v = zz;
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
    const float xend = mul2(K.pm_hi[8], K.pm_lo[8], xl, zz);
    return __shfl_sync(FULL, xend, 31);
}

// Joint scan of X and Y = dX/da over one segment, for the derivative in tau.  The pair obeys
//   X[t+1] = a X[t] + S[t],   Y[t+1] = a Y[t] + X[t],
// so a block of m bins maps (X, Y) to (a^m X + bx, a^m Y + m a^(m-1) X + by).  (xs, ys) = (X, Y)[t0];
// out_y[m] = Y[t0 + 8 lane + m]; returns (X, Y)[t0 + 256] through *xe, *ye (all lanes).
__device__ __forceinline__ void seg_scan_xy(const ScanConsts& K, float xs, float ys, uint32_t bits8, int lane,
                                            float pl_hi, float pl_lo, float pld_hi, float pld_lo, float out_y[8],
                                            float* xe, float* ye) {
    float zy[8];
    float ax = 0.f, ay = 0.f;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        zy[m] = ay;
        ay = mul2(K.a_hi, K.a_lo, ay, ax);
        ax = mul2(K.a_hi, K.a_lo, ax, (float)((bits8 >> m) & 1u));
    }
    // inclusive Kogge-Stone scan of (vx, vy) with block maps of 8 * 2^d bins
    float vx = ax, vy = ay;
#pragma unroll
    for (int d = 0; d < 5; ++d) {
        const float ox = __shfl_up_sync(FULL, vx, 1 << d);
        const float oy = __shfl_up_sync(FULL, vy, 1 << d);
        if (lane >= (1 << d)) {
            vy = mul2(K.ps_hi[d], K.ps_lo[d], oy, mul2(K.psd_hi[d], K.psd_lo[d], ox, vy));
            vx = mul2(K.ps_hi[d], K.ps_lo[d], ox, vx);
        }
    }
    float ex = __shfl_up_sync(FULL, vx, 1), ey = __shfl_up_sync(FULL, vy, 1);
    if (lane == 0) ex = ey = 0.f;
    // lane start: X_l = a^(8l) xs + ex,  Y_l = a^(8l) ys + 8l a^(8l-1) xs + ey
    const float xl = mul2(pl_hi, pl_lo, xs, ex);
    const float yl = mul2(pl_hi, pl_lo, ys, mul2(pld_hi, pld_lo, xs, ey));
#pragma unroll
    for (int m = 0; m < 8; ++m)
        out_y[m] = mul2(K.pm_hi[m], K.pm_lo[m], yl, mul2(K.pmd_hi[m], K.pmd_lo[m], xl, zy[m]));
    const float xend = mul2(K.pm_hi[8], K.pm_lo[8], xl, ax);
    const float yend = mul2(K.pm_hi[8], K.pm_lo[8], yl, mul2(K.pmd_hi[8], K.pmd_lo[8], xl, ay));
    *xe = __shfl_sync(FULL, xend, 31);
    *ye = __shfl_sync(FULL, yend, 31);
}

}  // namespace glm
