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
//   local part:   z_m = sum over this lane's spikes j < m of a^(m-1-j), each power rounded once.  (The
//                 recursion z_{m+1} = a z_m + S rounds the same chain 1, a, a^2, ... after every spike
//                 and so biases X by ~0.6 ulp; the direct powers do not.)
//   lane start:   X[t_lane] = a^(8 lane) x_seg + sum_{k < lane} a^(8 (lane - 1 - k)) z_8(k)
//                 (Kogge-Stone scan of the affine recurrence with constant multiplier a^8)
//   values:       X[t_lane + m] = a^m X[t_lane] + z_m
__device__ __forceinline__ float seg_scan(const ScanConsts& K, float x_seg, uint32_t bits8, float pl_hi,
                                          float pl_lo, int lane, float out[8]) {
    float z[8];
    float zz = 0.f;
    z[0] = 0.f;
#pragma unroll
    for (int m = 1; m <= 8; ++m) {  // static indices only: the powers stay in the constant bank
        float acc = 0.f;
#pragma unroll
        for (int j = 0; j < m; ++j) acc = fmaf((float)((bits8 >> j) & 1u), K.pr[m - 1 - j], acc);
        if (m < 8)
            z[m] = acc;
        else
            zz = acc;
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

}  // namespace glm
