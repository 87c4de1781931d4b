// Interval integrals of the continuous-time form (Sec. 2.3.2-2.3.3), shared by the U-product epilogue and
// the host entry point that exposes them for testing.
//
// Over one column [c_m, c_m + D) the potential relaxes as U(c_m + s) = b + u e^{-s/tau} (Eq. 8 between
// events), u = (W v)_i at the column start.  With a = exp(-D / tau), oma = 1 - a and rho = e^{-s/tau}:
//   F(u, D) - D = int_0^D (exp(u e^{-s/tau}) - 1) ds = tau int_a^1 expm1(u rho) / rho d rho
//               (the integral of Eq. 9; the paper evaluates it as tau (Ei(u) - Ei(u a)), Eq. 10)
//   G(u, D)     = int_0^D e^{-s/tau} exp(u e^{-s/tau}) ds = tau int_a^1 e^{u rho} d rho
//               (the interval weight of Eq. 14, tau (e^u - e^{u a}) / u)
// Both integrands are entire in rho, and w = |u| oma is how far the exponent moves over the column, so
// Gauss-Legendre quadrature in rho is accurate to FP32 with few nodes: 2 for w <= 0.1 (the usual case:
// columns are short against tau), 4 for w <= 1, else ceil(w) panels of 4 (at most 32).  Unlike the Ei
// difference it has no cancellation when a -> 1 and needs no division per element: the one-panel rules
// take the per-column factors q = tau oma w_k / (2 rho_k).
#pragma once

#include <math.h>

namespace glm {

// Gauss-Legendre nodes on [0, 1] (eta = (1 + xi) / 2) and weights on [-1, 1]
constexpr float GL2_E0 = 0.21132486540518712f, GL2_E1 = 0.78867513459481288f;
constexpr float GL4_E0 = 0.06943184420297371f, GL4_E1 = 0.33000947820757187f;
constexpr float GL4_E2 = 0.66999052179242813f, GL4_E3 = 0.93056815579702629f;
constexpr float GL4_W0 = 0.34785484513745386f, GL4_W1 = 0.65214515486254614f;
constexpr double GL2_E0D = 0.21132486540518712, GL2_E1D = 0.78867513459481288;
constexpr double GL4_E0D = 0.06943184420297371, GL4_E1D = 0.33000947820757187;
constexpr double GL4_E2D = 0.66999052179242813, GL4_E3D = 0.93056815579702629;
constexpr double GL4_W0D = 0.34785484513745386, GL4_W1D = 0.65214515486254614;
constexpr float CT_W2_MAX = 0.1f;   // largest |u| oma for the 2-node rule
constexpr int CT_PANELS_MAX = 32;

// Column constants, 8 floats: a, oma, q2[2], q4[4], from the column length D (FP64, then rounded).
__host__ __device__ __forceinline__ void ct_column(double D, double tau, float* col) {
    const double x = D / tau, a = exp(-x), oma = -expm1(-x);
    const double h = 0.5 * tau * oma;
    col[0] = (float)a;
    col[1] = (float)oma;
    col[2] = (float)(h / (a + oma * GL2_E0D));
    col[3] = (float)(h / (a + oma * GL2_E1D));
    col[4] = (float)(h * GL4_W0D / (a + oma * GL4_E0D));
    col[5] = (float)(h * GL4_W1D / (a + oma * GL4_E1D));
    col[6] = (float)(h * GL4_W1D / (a + oma * GL4_E2D));
    col[7] = (float)(h * GL4_W0D / (a + oma * GL4_E3D));
}

// e^x on the device's exp unit (ex2 of x log2 e, a few ulp), the C library's expf on the host.
__host__ __device__ __forceinline__ float ct_exp(float x) {
#ifdef __CUDA_ARCH__
    return __expf(x);
#else
    return expf(x);
#endif
}

// e^x and e^x - 1 of one node, branch-free: for |x| < 1/2 the Taylor series of e^x - 1 to x^8 (remainder
// below x^9 / 9!, i.e. 1.4e-8 relative), which keeps e^x - 1 exact near 0; otherwise e^x itself.
__host__ __device__ __forceinline__ void ct_node(float x, float* y, float* e) {
    const float p = x * fmaf(x, fmaf(x, fmaf(x, fmaf(x, fmaf(x, fmaf(x, fmaf(x, 1.f / 40320.f, 1.f / 5040.f),
                                                                        1.f / 720.f), 1.f / 120.f), 1.f / 24.f),
                                              1.f / 6.f), 0.5f), 1.f);
    const float ex = ct_exp(x);
    const bool small = fabsf(x) < 0.5f;
    *y = small ? p : ex - 1.f;
    *e = small ? 1.f + p : ex;
}

// The usual case (w = |u| oma <= 0.1), branch-free: dF = F(u, D) - D and eg = G(u, D) / tau by the
// 2-node rule, from the first four column constants {a, oma, q2[0], q2[1]}.  The nodes sit at m -+ z / u
// around the column midpoint m = a + oma / 2 (z = u oma / (2 sqrt 3), |z| <= 0.029), so one exponential
// at m and the series of e^{-+z} - 1 (even part z^2/2 (1 + z^2/12), odd part z (1 + z^2/6); remainder
// below z^5 / 120) give both: e^{u rho} - 1 = (e^{u m} - 1) + e^{u m} (e^{-+z} - 1).
__host__ __device__ __forceinline__ void ct_link2(float u, float a, float oma, float q0, float q1, float* dF,
                                                 float* eg) {
    float em1, em;
    ct_node(u * fmaf(oma, 0.5f, a), &em1, &em);
    const float z = u * oma * 0.28867513459481288f;
    const float z2 = z * z;
    const float ev = 0.5f * z2 * fmaf(z2, 1.f / 12.f, 1.f);
    const float od = z * fmaf(z2, 1.f / 6.f, 1.f);
    const float y0 = fmaf(em, ev - od, em1), y1 = fmaf(em, ev + od, em1);
    *dF = fmaf(q0, y0, q1 * y1);
    *eg = oma * em * (1.f + ev);
}

// Any element: dF = F(u, D) - D and eg = G(u, D) / tau = int_a^1 e^{u rho} d rho, from the column
// constants col = {a, oma, q2[2], q4[4]}.
__host__ __device__ __forceinline__ void ct_link(float u, const float* col, float tau, float* dF, float* eg) {
    const float a = col[0], oma = col[1];
    const float w = fabsf(u) * oma;
    if (w <= CT_W2_MAX) {
        ct_link2(u, a, oma, col[2], col[3], dF, eg);
    } else if (w <= 1.f) {
        float y0, y1, y2, y3, e0, e1, e2, e3;
        ct_node(u * fmaf(oma, GL4_E0, a), &y0, &e0);
        ct_node(u * fmaf(oma, GL4_E1, a), &y1, &e1);
        ct_node(u * fmaf(oma, GL4_E2, a), &y2, &e2);
        ct_node(u * fmaf(oma, GL4_E3, a), &y3, &e3);
        *dF = fmaf(col[4], y0, fmaf(col[5], y1, fmaf(col[6], y2, col[7] * y3)));
        *eg = 0.5f * oma * fmaf(GL4_W0, e0 + e3, GL4_W1 * (e1 + e2));
    } else {
        int P = (int)ceilf(w);
        if (P > CT_PANELS_MAX) P = CT_PANELS_MAX;
        const float h = oma / (float)P;
        float sf = 0.f, sg = 0.f;
        for (int p = 0; p < P; ++p) {
            const float base = fmaf((float)p, h, a);
            const float r0 = fmaf(h, GL4_E0, base), r1 = fmaf(h, GL4_E1, base);
            const float r2 = fmaf(h, GL4_E2, base), r3 = fmaf(h, GL4_E3, base);
            float y0, y1, y2, y3, e0, e1, e2, e3;
            ct_node(u * r0, &y0, &e0);
            ct_node(u * r1, &y1, &e1);
            ct_node(u * r2, &y2, &e2);
            ct_node(u * r3, &y3, &e3);
            sf += GL4_W0 * (y0 / r0 + y3 / r3) + GL4_W1 * (y1 / r1 + y2 / r2);
            sg += GL4_W0 * (e0 + e3) + GL4_W1 * (e1 + e2);
        }
        *dF = 0.5f * tau * h * sf;
        *eg = 0.5f * h * sg;
    }
}

// -ln(1 - x) for 0 <= x <= 0.1 by its series to x^7 / 7 (remainder below 1.5e-8 of the value)
__host__ __device__ __forceinline__ float ct_nlog1m(float x) {
    return x * fmaf(x, fmaf(x, fmaf(x, fmaf(x, fmaf(x, fmaf(x, 1.f / 7.f, 1.f / 6.f), 0.2f), 0.25f), 1.f / 3.f),
                       0.5f), 1.f);
}

// The explicit tau-derivative of one column's integral at fixed u (for dL/dtau):
//   T(u, D) = dF/dtau at fixed u = (F - D e^{u a}) / tau = u int_a^1 e^{u rho} (-ln rho) d rho
// (by parts from F = int_0^D exp(u e^{-s/tau}) ds; the second form by rho = e^{-s/tau}).  For a short
// column (oma <= 0.1) the first form cancels to ~oma of its terms, so the integral is taken by Gauss-Legendre
// quadrature in x = 1 - rho over [0, oma], with -ln rho = ct_nlog1m(x): 2 nodes where the exponent moves by
// |u| oma <= 0.1 (the usual case), 4 where it moves by at most 1, else panels of 4 (as in ct_link).  For
// oma > 0.1 the first form loses less than a digit.  dF = F - D from ct_link; D from the column constants
// (ct_length; not needed where u a = 0: then F - D e^{ua} = dF).
__host__ __device__ __forceinline__ float ct_length(float a, float oma, float tau) {
    if (oma <= 0.1f) return tau * ct_nlog1m(oma);
    return a < 0.5f ? -tau * logf(a) : -tau * log1pf(-oma);  // each form where its argument is exact
}
__host__ __device__ __forceinline__ float ct_dtau(float u, float a, float oma, float tau, float dF) {
    if (oma > 0.1f) {
        const float ua = u * a;
        if (ua == 0.f) return dF / tau;
        return (dF - ct_length(a, oma, tau) * expm1f(ua)) / tau;
    }
    const float w = fabsf(u) * oma;
    if (w <= CT_W2_MAX) {  // nodes at rho = a + oma eta, i.e. x = oma (1 - eta)
        const float x0 = oma * GL2_E1, x1 = oma * GL2_E0;
        return u * 0.5f * oma * (ct_exp(u - u * x0) * ct_nlog1m(x0) + ct_exp(u - u * x1) * ct_nlog1m(x1));
    }
    int P = (w <= 1.f) ? 1 : (int)ceilf(w);
    if (P > CT_PANELS_MAX) P = CT_PANELS_MAX;
    const float h = oma / (float)P;
    float sum = 0.f;
    for (int p = 0; p < P; ++p) {
        const float x0 = h * ((float)p + GL4_E0), x1 = h * ((float)p + GL4_E1);
        const float x2 = h * ((float)p + GL4_E2), x3 = h * ((float)p + GL4_E3);
        sum += GL4_W0 * (ct_exp(u - u * x0) * ct_nlog1m(x0) + ct_exp(u - u * x3) * ct_nlog1m(x3)) +
               GL4_W1 * (ct_exp(u - u * x1) * ct_nlog1m(x1) + ct_exp(u - u * x2) * ct_nlog1m(x2));
    }
    return u * 0.5f * h * sum;
}

}  // namespace glm
