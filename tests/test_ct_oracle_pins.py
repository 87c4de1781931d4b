"""Pins of the continuous-time oracle (oracle.continuous) to results it does not compute itself.

* Adaptive quadrature (scipy.integrate.quad) of exp(U_i(t)) between consecutive arrivals, with U built
  straight from its definition (Eq. 3: a sum over every earlier arrival, no recurrence, no Ei), and the
  spike part summed from the same definition: checks the recurrence (Eq. 8) and the Ei form (Eq. 10).
  Includes coincident spikes, a spike at t_begin, arrivals cut at t_end and a zero delay.
* Quadrature of exp(U_i) v_j for the integral part of the gradient (Eq. 14), and central finite
  differences of the oracle's own L for dL/dW and dL/db.
* Grid-aligned times with the delay equal to the bin width: U at the spike times equals the grid form
  b + W X at the spike bins (the grid oracle's filter, Eq. 13 on the grid); the grid log-likelihood is
  the left Riemann sum of the same integral, so L_grid - L_ct shrinks in proportion to the bin width.
* No spikes: L = -e^b (t_end - t_begin), dL/dW = 0.  A row without input (U = b, the u = 0 limit of
  Eq. 10 and 14): L_i and the integral part of dL/dW_ij in closed form.
"""
import numpy as np
import pytest
from scipy.integrate import quad

import oracle
from oracle import continuous as oc


def small_case(seed, n=3, t_end=0.4, rate=25.0, delay=0.0015, tau=0.02):
    rng = np.random.default_rng(seed)
    rows = []
    for i in range(n):
        k = rng.poisson(rate * t_end)
        rows.append(np.sort(rng.uniform(0.0, t_end, k)))
    # coincident spikes of two rows, a spike at t_begin, a spike whose arrival falls past t_end
    rows[0] = np.unique(np.append(rows[0], [0.0, 0.1234, t_end - 0.0005]))
    rows[1] = np.unique(np.append(rows[1], [0.1234]))
    offs = np.zeros(n + 1, dtype=np.int64)
    offs[1:] = np.cumsum([len(r) for r in rows])
    times = np.concatenate(rows)
    W = rng.normal(0.0, 1.0, (n, n))
    b = np.log(rng.uniform(5.0, 20.0, n))
    return offs, times, 0.0, t_end, tau, delay, W, b


def u_direct(offs, times, tau, delay, W, b, i, t):
    """Eq. 3 summed over every arrival at or before t."""
    s = b[i]
    for j in range(len(offs) - 1):
        a = times[offs[j]:offs[j + 1]] + delay
        a = a[a <= t]
        s += W[i, j] * np.exp(-(t - a) / tau).sum()
    return s


def v_direct(offs, times, tau, delay, j, t):
    a = times[offs[j]:offs[j + 1]] + delay
    a = a[a <= t]
    return np.exp(-(t - a) / tau).sum()


def breakpoints(times, t_begin, t_end, delay):
    arr = times + delay
    return np.unique(np.concatenate([[t_begin, t_end], arr[(arr > t_begin) & (arr < t_end)]]))


@pytest.mark.parametrize("seed,delay", [(0, 0.0015), (1, 0.0), (2, 0.004)])
def test_loglik_matches_quadrature(seed, delay):
    offs, times, t0, t1, tau, d, W, b = small_case(seed, delay=delay)
    r = oc.loglik_grad(offs, times, t0, t1, tau, d, W, b)
    bp = breakpoints(times, t0, t1, d)
    n = len(b)
    for i in range(n):
        integ = 0.0
        for lo, hi in zip(bp[:-1], bp[1:]):
            # the integrand on (lo, hi) includes the arrivals at lo (H(0) = 1) and none at hi
            f = lambda t: np.exp(u_direct(offs, times, tau, d, W, b, i, min(max(t, lo), hi - 1e-15 * hi)))
            integ += quad(f, lo, hi, epsabs=0.0, epsrel=1e-13, limit=200)[0]
        spk = sum(u_direct(offs, times, tau, d, W, b, i, t) for t in times[offs[i]:offs[i + 1]])
        L = spk - integ
        assert r["L"][i] == pytest.approx(L, rel=1e-11, abs=1e-11), (i, r["L"][i], L)
        assert r["integ"][i] == pytest.approx(integ, rel=1e-11)


def test_gradient_matches_quadrature_and_differences():
    offs, times, t0, t1, tau, d, W, b = small_case(3, n=3, t_end=0.3)
    r = oc.loglik_grad(offs, times, t0, t1, tau, d, W, b)
    bp = breakpoints(times, t0, t1, d)
    # Eq. 12: spike part and integral part of dL/dW_ij from their definitions
    for i, j in [(0, 0), (0, 2), (2, 1)]:
        spk = sum(v_direct(offs, times, tau, d, j, t) for t in times[offs[i]:offs[i + 1]])
        gi = 0.0
        for lo, hi in zip(bp[:-1], bp[1:]):
            def f(t):
                tt = min(max(t, lo), hi - 1e-15 * hi)
                return np.exp(u_direct(offs, times, tau, d, W, b, i, tt)) * v_direct(offs, times, tau, d, j, tt)
            gi += quad(f, lo, hi, epsabs=0.0, epsrel=1e-13, limit=200)[0]
        assert r["G"][i, j] == pytest.approx(spk - gi, rel=1e-10, abs=1e-10)
        assert r["C"][i, j] == pytest.approx(spk, rel=1e-12, abs=1e-14)
    # central finite differences of L in every W entry and b
    h = 1e-6
    n = len(b)
    for i in range(n):
        for j in range(n):
            Wp, Wm = W.copy(), W.copy()
            Wp[i, j] += h
            Wm[i, j] -= h
            fd = (oc.loglik_grad(offs, times, t0, t1, tau, d, Wp, b, grad=False)["L"][i]
                  - oc.loglik_grad(offs, times, t0, t1, tau, d, Wm, b, grad=False)["L"][i]) / (2 * h)
            assert r["G"][i, j] == pytest.approx(fd, rel=1e-6, abs=1e-6)
        bp_, bm_ = b.copy(), b.copy()
        bp_[i] += h
        bm_[i] -= h
        fd = (oc.loglik_grad(offs, times, t0, t1, tau, d, W, bp_, grad=False)["L"][i]
              - oc.loglik_grad(offs, times, t0, t1, tau, d, W, bm_, grad=False)["L"][i]) / (2 * h)
        assert r["gb"][i] == pytest.approx(fd, rel=1e-6, abs=1e-6)


def test_no_spikes_closed_form():
    n = 4
    offs = np.zeros(n + 1, dtype=np.int64)
    times = np.zeros(0)
    W = np.ones((n, n))
    b = np.log(np.array([1.0, 2.0, 5.0, 10.0]))
    r = oc.loglik_grad(offs, times, 1.0, 3.5, 0.01, 0.001, W, b)
    assert np.allclose(r["L"], -np.exp(b) * 2.5, rtol=1e-15)
    assert np.all(r["G"] == 0.0)
    assert np.allclose(r["gb"], -np.exp(b) * 2.5, rtol=1e-15)


def grid_case(n_bins, dt, seed=5, n=6):
    rng = np.random.default_rng(seed)
    rows = [np.sort(rng.choice(n_bins - 1, size=rng.integers(20, 60), replace=False)) for _ in range(n)]
    offs = np.zeros(n + 1, dtype=np.int64)
    offs[1:] = np.cumsum([len(r) for r in rows])
    bins = np.concatenate(rows).astype(np.int32)
    W = rng.normal(0.0, 0.8, (n, n))
    b = np.log(rng.uniform(5.0, 20.0, n))
    return offs, bins, W, b


def test_grid_aligned_times_reduce_to_the_grid_form():
    # a power-of-two bin width: bin * dt + dt is exactly (bin + 1) * dt, so an arrival one bin after a
    # spike lands on the next bin's spike time exactly, as on the grid
    dt, tau, n_bins = 2.0 ** -9, 0.02, 400
    offs, bins, W, b = grid_case(n_bins, dt)
    times = bins.astype(np.float64) * dt
    n = len(b)
    # U at the spike times equals b + W X at the spike bins (grid filter with a one-bin delay)
    X = oracle.filter(offs, bins, n_bins, dt, tau)
    for i in range(n):
        tb = bins[offs[i]:offs[i + 1]]
        u_ct = oc.u_at(offs, times, 0.0, n_bins * dt, tau, dt, W, b, tb * dt)[i]
        u_grid = b[i] + W[i] @ X[:, tb]
        assert np.allclose(u_ct, u_grid, rtol=1e-12, atol=1e-12)
    # the grid integral is the left Riemann sum: the gap shrinks with the bin width (same spike times,
    # bins split r ways, delay one bin = dt / r on both sides)
    gaps = []
    for r in (1, 2, 4, 8):
        g = oracle.loglik_grad(offs, (bins * r).astype(np.int32), n_bins * r, dt / r, tau, W, b)
        c = oc.loglik_grad(offs, times, 0.0, n_bins * dt, tau, dt / r, W, b, grad=False)
        gaps.append(abs(g["L_total"] - c["L_total"]))
    assert gaps[1] < 0.6 * gaps[0] and gaps[2] < 0.6 * gaps[1] and gaps[3] < 0.6 * gaps[2], gaps
    assert gaps[3] < 0.2 * gaps[0], gaps


def test_row_without_input_closed_form():
    """A row whose weights are all zero keeps U = b: L_i = q_i b_i - e^{b_i} (t_end - t_begin), and the
    integral part of dL/dW_ij is e^{b_i} int v_j dt = e^{b_i} tau sum_k (1 - exp(-(t_end - e_jk) / tau))."""
    offs, times, t0, t1, tau, d, W, b = small_case(4, n=3)
    W[1, :] = 0.0
    r = oc.loglik_grad(offs, times, t0, t1, tau, d, W, b)
    q1 = offs[2] - offs[1]
    assert r["L"][1] == pytest.approx(q1 * b[1] - np.exp(b[1]) * (t1 - t0), rel=1e-13)
    for j in range(3):
        e = times[offs[j]:offs[j + 1]] + d
        e = e[e < t1]
        integ = np.exp(b[1]) * tau * np.sum(1.0 - np.exp(-(t1 - e) / tau))
        assert r["C"][1, j] - r["G"][1, j] == pytest.approx(integ, rel=1e-12)


def quad_loglik(offs, times, t0, t1, tau, d, W, b, i):
    """L_i from its definition: the spike part from Eq. 3 at each spike, the integral by adaptive quadrature
    between the arrival breakpoints."""
    bp = breakpoints(times, t0, t1, d)
    integ = 0.0
    for lo, hi in zip(bp[:-1], bp[1:]):
        f = lambda t: np.exp(u_direct(offs, times, tau, d, W, b, i, min(max(t, lo), hi - 1e-15 * hi)))
        integ += quad(f, lo, hi, epsabs=0.0, epsrel=1e-13, limit=200)[0]
    spk = sum(u_direct(offs, times, tau, d, W, b, i, t) for t in times[offs[i]:offs[i + 1]])
    return spk - integ


@pytest.mark.parametrize("seed,delay", [(4, 0.0015), (5, 0.0)])
def test_dtau_matches_differences_of_the_definition(seed, delay):
    """dL_i/dtau against central differences (h = 1e-4 tau) of L_i computed from the model's definition
    (quadrature, not the oracle's recurrence), and against differences of the oracle's own L at a finer
    step; W = 0 makes U = b flat, so dL/dtau = 0."""
    offs, times, t0, t1, tau, d, W, b = small_case(seed, t_end=0.3, delay=delay)
    r = oc.loglik_grad(offs, times, t0, t1, tau, d, W, b)
    scale = np.abs(r["gtau_rows"]).sum()
    h = 1e-4 * tau
    for i in range(len(b)):
        fd = (quad_loglik(offs, times, t0, t1, tau + h, d, W, b, i)
              - quad_loglik(offs, times, t0, t1, tau - h, d, W, b, i)) / (2 * h)
        assert r["gtau_rows"][i] == pytest.approx(fd, rel=1e-6, abs=1e-7 * scale), (i, r["gtau_rows"][i], fd)
    h = 1e-6 * tau
    fd = (oc.loglik_grad(offs, times, t0, t1, tau + h, d, W, b, grad=False)["L"]
          - oc.loglik_grad(offs, times, t0, t1, tau - h, d, W, b, grad=False)["L"]) / (2 * h)
    assert np.all(np.abs(r["gtau_rows"] - fd) <= 1e-8 * scale)
    assert r["gtau"] == pytest.approx(r["gtau_rows"].sum(), rel=1e-15)
    z = oc.loglik_grad(offs, times, t0, t1, tau, d, np.zeros_like(W), b)
    assert np.all(z["gtau_rows"] == 0.0)
