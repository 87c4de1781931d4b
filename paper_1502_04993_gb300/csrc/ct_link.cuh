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

// e^x and e^x - 1 of one node: expm1 keeps e^x - 1 exact near 0; below x = -1 e^x comes from exp itself,
// where 1 + expm1 would keep none of its digits.
__host__ __device__ __forceinline__ void ct_node(float x, float* y, float* e) {
    *y = expm1f(x);
    *e = (x < -1.f) ? expf(x) : 1.f + *y;
}

// One element: dF = F(u, D) - D and gm = G(u, D) / (tau oma) = (1/oma) int_a^1 e^{u rho} d rho, from the
// column constants col = {a, oma, q2[2], q4[4]}.
__host__ __device__ __forceinline__ void ct_link(float u, const float* col, float tau, float* dF, float* gm) {
    const float a = col[0], oma = col[1];
    const float w = fabsf(u) * oma;
    if (w <= CT_W2_MAX) {
        float y0, y1, e0, e1;
        ct_node(u * fmaf(oma, GL2_E0, a), &y0, &e0);
        ct_node(u * fmaf(oma, GL2_E1, a), &y1, &e1);
        *dF = fmaf(col[2], y0, col[3] * y1);
        *gm = 0.5f * (e0 + e1);
    } else if (w <= 1.f) {
        float y0, y1, y2, y3, e0, e1, e2, e3;
        ct_node(u * fmaf(oma, GL4_E0, a), &y0, &e0);
        ct_node(u * fmaf(oma, GL4_E1, a), &y1, &e1);
        ct_node(u * fmaf(oma, GL4_E2, a), &y2, &e2);
        ct_node(u * fmaf(oma, GL4_E3, a), &y3, &e3);
        *dF = fmaf(col[4], y0, fmaf(col[5], y1, fmaf(col[6], y2, col[7] * y3)));
        *gm = 0.5f * fmaf(GL4_W0, e0 + e3, GL4_W1 * (e1 + e2));
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
        *gm = 0.5f * sg / (float)P;
    }
}

}  // namespace glm
