"""The continuous-time column integrals of the library (glm_ct_interval: the same FP32 code as the
U-product epilogue, run on the host) against their closed forms: F = tau (Ei(u) - Ei(u a)) (Eq. 10) and
G = tau (e^u - e^{u a}) / u (Eq. 14), evaluated with mpmath at 40 digits (the FP64 Ei difference loses
its digits to cancellation on short columns), across the 2-node, 4-node and multi-panel regimes of the
quadrature, short and long columns, u of either sign and u = 0."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def glm():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1502_04993_gb300 as g
    return g


def exact(u, D, tau):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    u_, D_, t_ = mp.mpf(u), mp.mpf(D), mp.mpf(tau)
    a = mp.exp(-D_ / t_)
    if u == 0.0:
        return float(D_), float(t_ * (1 - a))
    return float(t_ * (mp.ei(u_) - mp.ei(u_ * a))), float(t_ * (mp.exp(u_) - mp.exp(u_ * a)) / u_)


@pytest.mark.parametrize("x", [1e-7, 1e-4, 0.0125, 0.1, 0.7, 3.0, 25.0, 800.0])
@pytest.mark.parametrize("u", [0.0, 1e-6, -1e-3, 0.3, -0.9, 2.5, -4.0, 9.0, -25.0, 40.0, -150.0])
def test_interval_integrals(glm, u, x):
    tau = 0.01
    D = x * tau
    F, G = glm.ct_interval(u, D, tau)
    Fe, Ge = exact(u, D, tau)
    # FP32 arithmetic on u rho and expm1: ~1e-6 of the part beyond D (F - D), of F, and of G
    w = abs(u) * -np.expm1(-x)
    tolF = 2e-6 * (abs(Fe - D) * (1 + abs(u)) + 1e-6 * Fe) + (3e-6 * abs(Fe - D) if w > 1 else 0.0)
    assert abs(F - Fe) <= tolF + 1e-300, (u, x, F, Fe)
    # G relative to its own size, down to the FP32 underflow of e^{u rho} (u = -150)
    assert abs(G - Ge) <= 3e-6 * (1 + abs(u)) * Ge + 1e-37 * D, (u, x, G, Ge)


def test_interval_rejects_bad_input(glm):
    for args in [(0.0, -1.0, 0.01), (0.0, 1.0, 0.0), (np.nan, 1.0, 0.01)]:
        with pytest.raises(glm.GLMError):
            glm.ct_interval(*args)


def exact_dtau(u, D, tau):
    """dF/dtau at fixed u = (F - D e^{u a}) / tau, and F - D, at 40 digits."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    u_, D_, t_ = mp.mpf(u), mp.mpf(D), mp.mpf(tau)
    a = mp.exp(-D_ / t_)
    if u == 0.0:
        return 0.0, 0.0
    F = t_ * (mp.ei(u_) - mp.ei(u_ * a))
    return float((F - D_ * mp.exp(u_ * a)) / t_), float(F - D_)


@pytest.mark.parametrize("x", [1e-7, 1e-4, 0.0125, 0.1, 0.105, 0.2, 0.7, 3.0, 25.0, 800.0])
@pytest.mark.parametrize("u", [0.0, 1e-6, -1e-3, 0.3, -0.9, 2.5, -4.0, 9.0, -25.0, 40.0, -150.0])
def test_interval_tau_derivative(glm, u, x):
    """The explicit tau-derivative of F (glm_ct_interval_dtau: quadrature in 1 - rho for 1 - a <= 0.1, the
    closed form beyond) against the closed form at 40 digits.  Its FP32 error is measured against the size
    of the terms it is formed from, |T| + |F - D| / tau, times 1 + |u| (the relative error of e^{u rho} in
    FP32 grows with |u|): the closed form just above 1 - a = 0.1 cancels to ~1 - a of those terms."""
    tau = 0.01
    D = x * tau
    T = glm.ct_interval_dtau(u, D, tau)
    Te, dFe = exact_dtau(u, D, tau)
    assert abs(T - Te) <= 2e-6 * (abs(Te) + abs(dFe) / tau) * (1 + abs(u)) + 1e-30, (u, x, T, Te)
