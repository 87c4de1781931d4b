// e^v - 1 of an FP32 argument, rounded once to FP32 from a double-float value (~40 significant bits), for
// the link epilogue of the plain FP32 form (Eq. 5: the rate e^U = e^b e^v enters the integral of Eq. 7 as
// e^b (1 + (e^v - 1))).  A rounding error of the exponential that is biased by a few hundredths of an ulp on
// average shifts the integral term of L by ~1e-9 relative, the whole error budget of that form; this
// evaluation is correctly rounded but for rare near-ties, so its mean error is ~0.
//
// Method (written from the mathematics): Cody-Waite argument reduction v = k ln2 + r, |r| <= ln2 / 2, with
// ln2 split as LN2_HI (16 significant bits, so k LN2_HI and v - k LN2_HI are exact) + LN2_LO; then the
// Taylor series of e^r - 1 = r + r^2/2 + r^3/6 + r^4 Q(r), Q up to r^5 / 9! (truncation below 2^-38 of the
// result), the first three terms in double-float and r^4 Q(r) (at most 6.3e-4) in FP32; finally
// e^v - 1 = 2^k (1 + (e^r - 1)) - 1 in double-float.
//
// Host and device give the same bits: every product that is added is an explicit fused multiply-add and
// every other operation is explicitly rounded, so no compiler contraction changes the sequence.
#pragma once

#include <cmath>

namespace glm {

namespace ex1 {
#ifdef __CUDA_ARCH__
__device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
#else
inline float mul(float a, float b) {
    volatile float p = a * b;
    return p;
}
inline float add(float a, float b) {
    volatile float s = a + b;
    return s;
}
inline float sub(float a, float b) {
    volatile float s = a - b;
    return s;
}
#endif

struct df {
    float h, l;
};

// Knuth's TwoSum, then the low parts added: h + l = a.h + a.l + b.h + b.l to ~2^-44 relative
__host__ __device__ inline df dadd(df a, df b) {
    const float s = add(a.h, b.h);
    const float bp = sub(s, a.h);
    float e = add(sub(a.h, sub(s, bp)), sub(b.h, bp));
    e = add(e, add(a.l, b.l));
    const float h = add(s, e);
    return df{h, sub(e, sub(h, s))};
}
// product with the exact error term of a.h b.h from a fused multiply-add
__host__ __device__ inline df dmul(df a, df b) {
    const float p = mul(a.h, b.h);
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, fmaf(a.l, b.h, e));
    const float h = add(p, e);
    return df{h, sub(e, sub(h, p))};
}
}  // namespace ex1

__host__ __device__ inline float expm1_acc(float v) {
    using namespace ex1;
    if (v != v) return v;
    if (v > 88.72f) return INFINITY;   // e^v beyond FP32
    if (v < -20.f) return -1.f;        // e^v < 2^-28: e^v - 1 rounds to -1
    const float LN2_HI = 0.693145751953125f;        // 45426 / 2^16
    const float LN2_LO = 1.4286068203094173e-06f;   // ln 2 - LN2_HI
    const float k = rintf(mul(v, 1.44269504088896341f));
    // v - k ln2 (the first part exact), normalised to a pair with |l| <= ulp(h) / 2 (dmul drops l l)
    const df r = dadd(df{fmaf(-k, LN2_HI, v), 0.f}, df{mul(-k, LN2_LO), 0.f});
    const float rf = r.h;
    // r^4 Q(r) = r^4 (1/24 + r/120 + r^2/720 + r^3/5040 + r^4/40320 + r^5/362880)
    float q = 2.7557319223985893e-06f;
    q = fmaf(q, rf, 2.4801587301587302e-05f);
    q = fmaf(q, rf, 1.9841269841269841e-04f);
    q = fmaf(q, rf, 1.3888888888888889e-03f);
    q = fmaf(q, rf, 8.3333333333333333e-03f);
    q = fmaf(q, rf, 4.1666666666666667e-02f);
    const float r2f = mul(rf, rf);
    const float t4 = mul(mul(r2f, r2f), q);
    // r + r^2 / 2 + r^3 / 6 in double-float
    const df r2 = dmul(r, r);
    const df r3 = dmul(r2, r);
    const df sixth{0.16666667163372040f, -4.9670539e-09f};  // 1/6 as hi + lo
    df m = dadd(r, df{mul(r2.h, 0.5f), mul(r2.l, 0.5f)});
    m = dadd(m, dmul(r3, sixth));
    m = dadd(m, df{t4, 0.f});
    if (k == 0.f) return add(m.h, m.l);
    // e^v - 1 = 2^k m + (2^k - 1), both parts exact scalings / sums in double-float
    const int ki = (int)k;
    const df scaled{ldexpf(m.h, ki), ldexpf(m.l, ki)};
    const df c = dadd(df{ldexpf(1.f, ki), 0.f}, df{-1.f, 0.f});
    const df res = dadd(scaled, c);
    return add(res.h, res.l);
}

}  // namespace glm
