"""Pins of the per-row tau / delay oracle (oracle.delays) to results it does not compute itself.

* One class with the one-bin delay: equal to the loop-based grid oracle (oracle.loglik_grad, C).
* A tiny network with three different (tau_i, d_i): U, L, dL/dW and dL/db straight from the definition
  (a sum over every earlier spike with its own delay and time constant; no filter, no recursion).
* Central finite differences of its own L in W and b.
* A delay that pushes spikes past the recording: those spikes contribute nothing.
"""
import numpy as np
import pytest

import oracle
from oracle import delays as od


def tiny(seed, n=3, T=80):
    rng = np.random.default_rng(seed)
    rows = [np.sort(rng.choice(T, size=rng.integers(4, 10), replace=False)) for _ in range(n)]
    offs = np.zeros(n + 1, dtype=np.int64)
    offs[1:] = np.cumsum([len(r) for r in rows])
    bins = np.concatenate(rows).astype(np.int32)
    W = rng.normal(0.0, 0.8, (n, n))
    b = np.log(rng.uniform(5.0, 20.0, n))
    return offs, bins, W, b


def direct(offs, bins, T, dt, taus, ds, W, b, selfd=None):
    """Definition: U_i[t] = b_i + sum_j W_ij sum_{s: s + D_ij <= t} exp(-(t - D_ij - s) dt / tau_i), with
    D_ij = d_i for j != i and D_ii = the self-delay (d_i unless given)."""
    n = len(offs) - 1
    selfd = ds if selfd is None else selfd
    L, G, gb = np.zeros(n), np.zeros((n, n)), np.zeros(n)
    for i in range(n):
        X = np.zeros((n, T))
        for j in range(n):
            dij = selfd[i] if j == i else ds[i]
            for s in bins[offs[j]:offs[j + 1]]:
                for t in range(s + dij, T):
                    X[j, t] += np.exp(-(t - dij - s) * dt / taus[i])
        U = b[i] + W[i] @ X
        S = np.zeros(T)
        S[bins[offs[i]:offs[i + 1]]] = 1.0
        R = S - dt * np.exp(U)
        L[i] = (S * U).sum() - dt * np.exp(U).sum()
        G[i] = X @ R
        gb[i] = R.sum()
    return L, G, gb


def test_one_class_with_unit_delay_is_the_grid_oracle():
    offs, bins, W, b = tiny(0, n=5, T=300)
    r = od.loglik_grad_classes(offs, bins, 300, 0.001, [0.01] * 5, [1] * 5, W, b)
    g = oracle.loglik_grad(offs, bins, 300, 0.001, 0.01, W, b)
    assert np.allclose(r["L"], g["L"], rtol=1e-12, atol=1e-12)
    assert np.allclose(r["G"], g["G"], rtol=1e-10, atol=1e-12)
    assert np.allclose(r["gb"], g["gb"], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("seed", [1, 2])
def test_classes_match_the_definition(seed):
    T, dt = 80, 0.002
    offs, bins, W, b = tiny(seed, T=T)
    taus, ds = [0.008, 0.02, 0.012], [1, 3, 6]
    r = od.loglik_grad_classes(offs, bins, T, dt, taus, ds, W, b)
    L, G, gb = direct(offs, bins, T, dt, taus, ds, W, b)
    assert np.allclose(r["L"], L, rtol=1e-12, atol=1e-12)
    assert np.allclose(r["G"], G, rtol=1e-11, atol=1e-12)
    assert np.allclose(r["gb"], gb, rtol=1e-12, atol=1e-12)


def test_classes_gradient_is_the_derivative():
    T, dt = 120, 0.001
    offs, bins, W, b = tiny(3, n=4, T=T)
    taus, ds = [0.01, 0.01, 0.015, 0.02], [2, 2, 1, 4]
    r = od.loglik_grad_classes(offs, bins, T, dt, taus, ds, W, b)
    h = 1e-6
    for i in range(4):
        for j in range(4):
            Wp, Wm = W.copy(), W.copy()
            Wp[i, j] += h
            Wm[i, j] -= h
            fd = (od.loglik_grad_classes(offs, bins, T, dt, taus, ds, Wp, b)["L"][i]
                  - od.loglik_grad_classes(offs, bins, T, dt, taus, ds, Wm, b)["L"][i]) / (2 * h)
            assert r["G"][i, j] == pytest.approx(fd, rel=1e-6, abs=1e-8)
        bp, bm = b.copy(), b.copy()
        bp[i] += h
        bm[i] -= h
        fd = (od.loglik_grad_classes(offs, bins, T, dt, taus, ds, W, bp)["L"][i]
              - od.loglik_grad_classes(offs, bins, T, dt, taus, ds, W, bm)["L"][i]) / (2 * h)
        assert r["gb"][i] == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_delay_past_the_recording():
    offs = np.array([0, 2, 3], dtype=np.int64)
    bins = np.array([10, 48, 30], dtype=np.int32)
    so, sb = od.shift_trains(offs, bins, 50, 4)
    assert so.tolist() == [0, 1, 2] and sb.tolist() == [14, 34]
    W = np.array([[0.5, -1.0], [2.0, 0.3]])
    b = np.log(np.array([10.0, 4.0]))
    r = od.loglik_grad_classes(offs, bins, 50, 0.001, [0.01, 0.01], [5, 5], W, b)
    L, G, gb = direct(offs, bins, 50, 0.001, [0.01, 0.01], [5, 5], W, b)
    assert np.allclose(r["L"], L, rtol=1e-12) and np.allclose(r["G"], G, rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("seed", [4, 5])
def test_self_delay_matches_the_definition(seed):
    """The paper's separate self-delay (Sec. 2.4, Sec. 3.1): the diagonal term acts after s_i bins, every other
    source after d_i; against the per-pair definition, including s_i = d_i rows (no change)."""
    T, dt = 90, 0.001
    offs, bins, W, b = tiny(seed, n=4, T=T)
    taus, ds, selfd = [0.01, 0.01, 0.015, 0.02], [3, 3, 2, 4], [1, 3, 1, 2]
    r = od.loglik_grad_classes(offs, bins, T, dt, taus, ds, W, b, self_delay_rows=selfd)
    L, G, gb = direct(offs, bins, T, dt, taus, ds, W, b, selfd=selfd)
    assert np.allclose(r["L"], L, rtol=1e-12, atol=1e-12)
    assert np.allclose(r["G"], G, rtol=1e-11, atol=1e-12)
    assert np.allclose(r["gb"], gb, rtol=1e-12, atol=1e-12)
    # and it differs from the uniform-delay model exactly where a self-delay differs
    u = od.loglik_grad_classes(offs, bins, T, dt, taus, ds, W, b)
    differ = np.array(selfd) != np.array(ds)
    assert np.all(np.abs(r["L"] - u["L"])[differ] > 1e-9) and np.array_equal(r["L"][~differ], u["L"][~differ])


def test_self_delay_gradient_is_the_derivative():
    T, dt = 100, 0.001
    offs, bins, W, b = tiny(6, n=3, T=T)
    taus, ds, selfd = [0.01, 0.012, 0.01], [2, 4, 3], [1, 1, 3]
    r = od.loglik_grad_classes(offs, bins, T, dt, taus, ds, W, b, self_delay_rows=selfd)
    h = 1e-6
    for i in range(3):
        Wp, Wm = W.copy(), W.copy()
        Wp[i, i] += h
        Wm[i, i] -= h
        fd = (od.loglik_grad_classes(offs, bins, T, dt, taus, ds, Wp, b, self_delay_rows=selfd)["L"][i]
              - od.loglik_grad_classes(offs, bins, T, dt, taus, ds, Wm, b, self_delay_rows=selfd)["L"][i]) / (2 * h)
        assert r["G"][i, i] == pytest.approx(fd, rel=1e-6, abs=1e-8)
