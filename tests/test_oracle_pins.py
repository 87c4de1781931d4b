"""Pins of the FP64 oracle to facts fixed outside it: closed forms, the paper's recursions, brute force
on tiny inputs, finite differences, the concavity theorem (App. A), recovery of a known network, and
the values the paper prints (App. C).  None of these re-types the oracle's own formula."""
import math
import os

import numpy as np
import pytest

import oracle
import synth
from oracle.classify import truth_labels

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def random_spikes(n, T, p, seed, *, min_per_row=0):
    rng = np.random.default_rng(seed)
    rows = []
    for i in range(n):
        s = np.flatnonzero(rng.random(T) < p)
        if s.size < min_per_row:
            s = np.unique(np.concatenate([s, rng.choice(T, min_per_row, replace=False)]))
        rows.append(s.astype(np.int32))
    offs = np.zeros(n + 1, dtype=np.int64)
    offs[1:] = np.cumsum([r.size for r in rows])
    bins = np.concatenate(rows) if offs[-1] else np.zeros(0, dtype=np.int32)
    return offs, bins, rows


# --------------------------------------------------------------------------- generator (inputs)

def test_philox_known_answers():
    for r in golden_rows("philox4x32_10_kat.txt"):
        v = [int(x, 16) for x in r]
        assert synth.philox4x32_10(v[0:4], v[4:6]) == tuple(v[6:10])


def test_generator_is_thread_count_independent():
    a = synth.make_workload("glm_n50_t20k", threads=1, n_bins=5000)
    b = synth.make_workload("glm_n50_t20k", threads=3, n_bins=5000)
    assert np.array_equal(a["offs"], b["offs"]) and np.array_equal(a["bins"], b["bins"])


def test_generator_network_structure():
    n, ne, p = 400, 320, 0.1
    W, types = synth.network(n, ne, p, 0.2, 0.8, seed=3)
    assert np.all(np.diag(W) == 0)
    assert np.all(types[:ne] == 1) and np.all(types[ne:] == -1)
    off = ~np.eye(n, dtype=bool)
    frac = (W[off] != 0).mean()
    assert abs(frac - p) < 4 * math.sqrt(p * (1 - p) / off.sum())
    # Dale's law by presynaptic column
    assert np.all(W[:, :ne][W[:, :ne] != 0] == 0.2)
    assert np.all(W[:, ne:][W[:, ne:] != 0] == -0.8)
    Ws, ts = synth.network(n, ne, p, 0.2, 0.8, seed=3, w_self=-6.25, syn_groups=3, syn_size=10, w_syn=0.3,
                           shuffle=True)
    assert np.all(np.diag(Ws) == -6.25) and (ts == 1).sum() == ne


# --------------------------------------------------------------------------- X, Eq. 13

def test_filter_equals_direct_convolution_sum():
    n, T, dt, tau = 3, 300, 1e-3, 7e-3
    a = math.exp(-dt / tau)
    offs, bins, rows = random_spikes(n, T, 0.05, 1)
    X = oracle.filter(offs, bins, T, dt, tau)
    for j in range(n):
        S = np.zeros(T)
        S[rows[j]] = 1
        for t in range(T):
            direct = 0.0
            for s in range(t):  # kernel H(t-s-1) e^{-(t-s-1) dt / tau}: causal, one-bin delay
                direct += a ** (t - 1 - s) * S[s]
            assert X[j, t] == pytest.approx(direct, rel=1e-13, abs=1e-300)


def test_filter_matches_event_recursion_of_eq13():
    """Just after each spike the filtered train satisfies v(t_{k+1}) = v(t_k) e^{-(t_{k+1}-t_k)/tau} + 1."""
    n, T, dt, tau = 2, 2000, 1e-3, 10e-3
    offs, bins, rows = random_spikes(n, T - 1, 0.02, 2)
    X = oracle.filter(offs, bins, T, dt, tau)
    for j in range(n):
        s = rows[j]
        for k in range(len(s) - 1):
            lhs = X[j, s[k + 1] + 1]
            rhs = X[j, s[k] + 1] * math.exp(-(s[k + 1] - s[k]) * dt / tau) + 1.0
            assert lhs == pytest.approx(rhs, rel=1e-12)


def test_filter_edge_cases():
    T, dt, tau = 10, 1e-3, 1e-2
    offs = np.array([0, 0, 1, 2], dtype=np.int64)  # row 0 silent, row 1 spikes at 0, row 2 at the last bin
    bins = np.array([0, T - 1], dtype=np.int32)
    X = oracle.filter(offs, bins, T, dt, tau)
    assert np.all(X[0] == 0)
    assert X[1, 0] == 0 and X[1, 1] == 1.0
    assert np.all(X[2] == 0)
    with pytest.raises(ValueError):
        oracle.filter(np.array([0, 2], dtype=np.int64), np.array([3, 3], dtype=np.int32), T, dt, tau)
    with pytest.raises(ValueError):
        oracle.filter(np.array([0, 1], dtype=np.int64), np.array([T], dtype=np.int32), T, dt, tau)


# --------------------------------------------------------------------------- L, G: closed forms

def test_closed_forms_at_zero_coupling():
    """W = 0: U_i = b_i, so L_i = q_i b_i - T dt e^{b_i}, dL/db_i = q_i - T dt e^{b_i} (Sec. 2.3.3: the bias
    is stationary when the expected count equals q_i), and dL/dW_ij is a sum over spike pairs minus a
    geometric series (Eq. 12 with Eq. 13)."""
    n, T, dt, tau = 4, 3000, 1e-3, 8e-3
    a = math.exp(-dt / tau)
    offs, bins, rows = random_spikes(n, T, 0.01, 3, min_per_row=1)
    b = np.array([0.3, 1.1, 2.0, -0.5])
    r = oracle.loglik_grad(offs, bins, T, dt, tau, np.zeros((n, n)), b)
    for i in range(n):
        q = len(rows[i])
        assert r["L"][i] == pytest.approx(q * b[i] - T * dt * math.exp(b[i]), rel=1e-12)
        assert r["gb"][i] == pytest.approx(q - T * dt * math.exp(b[i]), rel=1e-11, abs=1e-9)
        for j in range(n):
            pairs = sum(a ** (t - 1 - s) for t in rows[i] for s in rows[j] if s < t)
            geo = sum((1 - a ** (T - 1 - s)) / (1 - a) for s in rows[j])
            want = pairs - dt * math.exp(b[i]) * geo
            assert r["G"][i, j] == pytest.approx(want, rel=1e-10, abs=1e-10)
    assert r["gtau"] == 0.0


def test_single_neuron_self_coupling_closed_forms():
    """One neuron, one spike at bin s, self weight w.  At w = 0: dL/dw = -dt e^b (1 - a^{T-1-s}) / (1 - a)
    (the spike bin itself sees X = 0), d2L/dw2 = -dt e^b (1 - a^{2(T-1-s)}) / (1 - a^2)  (Eq. 18).  For any
    w the potential after the spike is b + w a^k."""
    T, dt, tau, s, b = 500, 1e-3, 5e-3, 120, math.log(30.0)
    a = math.exp(-dt / tau)
    offs = np.array([0, 1], dtype=np.int64)
    bins = np.array([s], dtype=np.int32)

    def L(w):
        return oracle.eval_rows(offs, bins, T, dt, tau, np.array([[w]]), np.array([b]))

    r0 = L(0.0)
    assert r0["G"][0, 0] == pytest.approx(-dt * math.exp(b) * (1 - a ** (T - 1 - s)) / (1 - a), rel=1e-12)
    h = 1e-3
    d2 = (L(h)["L"][0] - 2 * r0["L"][0] + L(-h)["L"][0]) / h ** 2
    assert d2 == pytest.approx(-dt * math.exp(b) * (1 - a ** (2 * (T - 1 - s))) / (1 - a * a), rel=1e-5)
    w = -1.7
    brute = b - dt * math.exp(b) * ((s + 1) + sum(math.exp(w * a ** k) for k in range(T - 1 - s)))
    assert L(w)["L"][0] == pytest.approx(brute, rel=1e-12)


def test_loglik_matches_potential_recursion_brute_force():
    """U from the leaky-integrator recursion (Eq. 4 / Eq. 8 on the grid) instead of b + W X."""
    n, T, dt, tau = 3, 400, 1e-3, 6e-3
    a = math.exp(-dt / tau)
    offs, bins, rows = random_spikes(n, T, 0.03, 4)
    rng = np.random.default_rng(5)
    W = rng.normal(0, 0.7, (n, n))
    b = rng.normal(1.5, 0.3, n)
    S = np.zeros((n, T))
    for j in range(n):
        S[j, rows[j]] = 1
    r = oracle.loglik_grad(offs, bins, T, dt, tau, W, b)
    for i in range(n):
        V, Li = 0.0, 0.0
        for t in range(T):
            if t > 0:
                V = a * V + sum(W[i, j] * S[j, t - 1] for j in range(n))
            U = b[i] + V
            Li += S[i, t] * U - dt * math.exp(U)
        assert r["L"][i] == pytest.approx(Li, rel=1e-12)


# --------------------------------------------------------------------------- derivatives

@pytest.fixture(scope="module")
def fd_problem():
    w = synth.make_workload("glm_n50_t20k", n=8, n_exc=6, n_bins=6000, seed=11)
    rng = np.random.default_rng(12)
    W = rng.normal(0.0, 0.3, (8, 8))
    b = np.log(5.0) + rng.normal(0, 0.2, 8)
    return w, W, b


def test_gradient_matches_central_differences(fd_problem):
    w, W, b = fd_problem
    args = (w["offs"], w["bins"], w["n_bins"], w["dt"], w["tau"])
    r = oracle.loglik_grad(*args, W, b)
    rng = np.random.default_rng(13)
    h = 1e-4
    for _ in range(16):
        i, j = rng.integers(0, 8, 2)
        Wp, Wm = W.copy(), W.copy()
        Wp[i, j] += h
        Wm[i, j] -= h
        fd = (oracle.eval_rows(*args, Wp, b, [i], grad=False)["L"][0]
              - oracle.eval_rows(*args, Wm, b, [i], grad=False)["L"][0]) / (2 * h)
        assert r["G"][i, j] == pytest.approx(fd, rel=1e-6, abs=1e-6)
    for i in range(3):
        bp, bm = b.copy(), b.copy()
        bp[i] += h
        bm[i] -= h
        fd = (oracle.eval_rows(*args, W, bp, [i], grad=False)["L"][0]
              - oracle.eval_rows(*args, W, bm, [i], grad=False)["L"][0]) / (2 * h)
        assert r["gb"][i] == pytest.approx(fd, rel=1e-6, abs=1e-6)


def test_tau_derivative_matches_central_differences(fd_problem):
    w, W, b = fd_problem
    tau = w["tau"]
    r = oracle.loglik_grad(w["offs"], w["bins"], w["n_bins"], w["dt"], tau, W, b)
    h = 1e-4 * tau
    Lp = oracle.loglik_grad(w["offs"], w["bins"], w["n_bins"], w["dt"], tau + h, W, b)["L_total"]
    Lm = oracle.loglik_grad(w["offs"], w["bins"], w["n_bins"], w["dt"], tau - h, W, b)["L_total"]
    assert r["gtau"] == pytest.approx((Lp - Lm) / (2 * h), rel=1e-6)


def test_concavity_and_hessian_quadratic_form(fd_problem):
    """App. A: x^T H x = -int lambda V^2 dt <= 0 (Eq. 19); on the grid -dt sum_t e^{U} (dU)^2."""
    w, W, b = fd_problem
    args = (w["offs"], w["bins"], w["n_bins"], w["dt"], w["tau"])
    X = oracle.filter(w["offs"], w["bins"], w["n_bins"], w["dt"], w["tau"])
    U = b[:, None] + W @ X
    L0 = oracle.loglik_grad(*args, W, b)["L_total"]
    rng = np.random.default_rng(14)
    h = 1e-3
    for _ in range(12):
        DW = rng.normal(0, 1, W.shape)
        Db = rng.normal(0, 1, b.shape)
        Lp = oracle.loglik_grad(*args, W + h * DW, b + h * Db)["L_total"]
        Lm = oracle.loglik_grad(*args, W - h * DW, b - h * Db)["L_total"]
        second = (Lp - 2 * L0 + Lm) / h ** 2
        dU = Db[:, None] + DW @ X
        quad = -w["dt"] * np.sum(np.exp(U) * dU ** 2)
        assert second <= 0
        assert second == pytest.approx(quad, rel=1e-4)


# --------------------------------------------------------------------------- fit

CHAIN_W = np.array([[-2.0, 0.0, 0.0, 0.0],
                    [1.0, -2.0, 0.0, 0.0],
                    [0.0, -1.0, -2.0, 0.0],
                    [0.0, 0.0, 0.8, -2.0]])


@pytest.fixture(scope="module")
def chain_fit():
    n, T, dt, tau = 4, 200_000, 1e-3, 1e-2
    b = np.full(n, math.log(20.0))
    offs, bins = synth.simulate(CHAIN_W, b, tau, dt, T, seed=21)
    f = oracle.fit(offs, bins, T, dt, tau, eta=1e-13, max_iter=300)
    return dict(n=n, T=T, dt=dt, tau=tau, b=b, offs=offs, bins=bins, fit=f)


def test_fit_recovers_known_directed_network(chain_fit):
    """The MLE is consistent (Sec. 3.1): the fitted weights sit within 4 standard errors of the generating
    ones, the standard errors from the inverse observed Fisher information -H (Eq. 18).  The network is a
    directed chain, so a transposed W or a shifted delay convention fails."""
    c = chain_fit
    f = c["fit"]
    assert np.all(f["status"] == oracle.FIT_CONVERGED)
    X = oracle.filter(c["offs"], c["bins"], c["T"], c["dt"], c["tau"])
    V = np.vstack([np.ones(c["T"]), X])  # v_i0 = 1, v_ij = X_j (Eq. 11)
    for i in range(c["n"]):
        theta = np.concatenate([[f["b"][i]], f["W"][i]])
        lam = np.exp(theta @ V)
        H = -(V * (c["dt"] * lam)) @ V.T
        se = np.sqrt(np.diag(np.linalg.inv(-H)))
        truth = np.concatenate([[c["b"][i]], CHAIN_W[i]])
        z = np.abs(theta - truth) / se
        assert np.all(z < 4.0), (i, z)


def test_fit_bias_stationarity(chain_fit):
    """At the maximum, the expected spike count equals the observed one, q_i = dt sum_t e^{U_i[t]} (Sec. 2.3.3)."""
    c = chain_fit
    r = oracle.loglik_grad(c["offs"], c["bins"], c["T"], c["dt"], c["tau"], c["fit"]["W"], c["fit"]["b"])
    q = np.diff(c["offs"])
    assert np.all(np.abs(r["gb"]) < 1e-6 * q)
    # the remaining gradient is tiny against the size of its two terms (both ~ q_i * mean X)
    assert np.all(np.abs(r["G"]) < 1e-7 * q[:, None])


def test_fit_methods_agree_and_degenerate_row():
    n, T, dt, tau = 3, 20_000, 1e-3, 1e-2
    W = np.array([[-1.0, 0.0, 0.0], [0.8, -1.0, 0.0], [0.0, 0.0, -1.0]])
    offs, bins = synth.simulate(W, np.full(n, math.log(15.0)), tau, dt, T, seed=5)
    # append a silent fourth neuron
    offs4 = np.concatenate([offs, [offs[-1]]]).astype(np.int64)
    f1 = oracle.fit(offs4, bins, T, dt, tau, method="lbfgs", eta=1e-14, max_iter=500)
    f2 = oracle.fit(offs4, bins, T, dt, tau, method="ga", eta=1e-14, max_iter=20000)
    assert f1["status"][3] == oracle.FIT_DEGENERATE and f1["b"][3] == pytest.approx(math.log(1e-3))
    assert np.all(f1["W"][3] == 0)
    assert np.allclose(f1["W"][:3], f2["W"][:3], atol=2e-3)
    assert np.allclose(f1["b"][:3], f2["b"][:3], atol=2e-3)
    assert f1["iters"][:3].max() < f2["iters"][:3].min()


# --------------------------------------------------------------------------- classification

def test_chance_level_mer_reproduces_printed_values():
    """A random classifier that keeps p and f_e misclassifies MER_0 of the pairs (Eq. 20); the paper prints
    33.28 % (p = 0.2) and 18.32 % (p = 0.1).  The oracle's MER applied to such a classifier must agree."""
    for p_s, fe_s, mer_s in golden_rows("mer0_printed.txt"):
        p, fe, mer0 = float(p_s), float(fe_s), float(mer_s)
        assert oracle.chance_mer(p, fe) == pytest.approx(mer0, abs=5e-5)
        n = 1000
        W, types = synth.network(n, int(fe * n), p, 1.0, 1.0, seed=7)
        truth = truth_labels(W)
        rng = np.random.default_rng(8)
        u = rng.random((n, n))
        lab = np.where(u < p * fe, 1, np.where(u < p, -1, 0)).astype(np.int8)
        np.fill_diagonal(lab, 0)
        got = oracle.mer_breakdown(lab, truth, types)["mer"]
        assert got == pytest.approx(mer0, abs=2.5e-3)


def test_classifiers_recover_separated_mixture():
    rng = np.random.default_rng(9)
    n = 120
    truth = rng.choice([-1, 0, 1], size=(n, n), p=[0.05, 0.8, 0.15]).astype(np.int8)
    np.fill_diagonal(truth, 0)
    W = np.where(truth == 1, 0.3, np.where(truth == -1, -1.2, 0.0)) + rng.normal(0, 0.03, (n, n))
    for method in ("kmeans", "gmm"):
        lab, model = oracle.classify(W, method)
        assert oracle.mer_breakdown(lab, truth)["errors"] == 0, method


def test_mer_breakdown_counts_by_hand():
    truth = np.array([[0, 1, -1], [0, 0, -1], [1, 0, 0]], dtype=np.int8)
    lab = np.array([[0, 0, -1], [1, 0, 1], [1, -1, 0]], dtype=np.int8)
    types = np.array([1, 1, -1])
    r = oracle.mer_breakdown(lab, truth, types)
    # off-diagonal pairs: (0,1) E->0 FN_E; (1,0) 0->E FP_E; (1,2) I->E FP_E + Dale violation; (2,1) 0->I FP_I
    assert r["errors"] == 4 and r["mer"] == pytest.approx(4 / 6) and r["mer_n2"] == pytest.approx(4 / 9)
    assert (r["exc"]["fp"], r["exc"]["fn"], r["exc"]["nd"]) == (2, 1, 1)
    assert (r["inh"]["fp"], r["inh"]["fn"], r["inh"]["nd"]) == (1, 1, 1)
    assert (r["absent"]["fp"], r["absent"]["fn"]) == (1, 2)


def test_l1_penalised_fit_stationarity_and_shrinkage():
    """Eq. 16-17: at the penalised optimum dL/dW_ij = alpha W_ij / sqrt(W_ij^2 + eps) for j != i, while the
    self weight and the bias are not penalised (dL/dW_ii = dL/db_i = 0); alpha = 0 is the plain fit; and the
    off-diagonal weights shrink as alpha grows.  The gradient comes from the evaluation routine, not from
    the fit's own objective."""
    w = synth.make_workload("glm_n50_t20k", n_bins=8000)
    args = (w["offs"], w["bins"], 8000, w["dt"], w["tau"])
    plain = oracle.fit(*args, eta=1e-13, max_iter=800)
    zero = oracle.fit(*args, eta=1e-13, max_iter=800, alpha=0.0)
    assert np.array_equal(plain["W"], zero["W"]) and np.array_equal(plain["b"], zero["b"])
    eps = 1e-4
    sums = []
    for alpha in (0.5, 2.0, 8.0):
        f = oracle.fit(*args, eta=1e-14, max_iter=2000, alpha=alpha, eps=eps)
        r = oracle.loglik_grad(*args, f["W"], f["b"])
        n = f["W"].shape[0]
        off = ~np.eye(n, dtype=bool)
        resid = r["G"] - alpha * f["W"] / np.sqrt(f["W"] ** 2 + eps)
        q = np.diff(w["offs"]).astype(np.float64)
        assert np.max(np.abs(resid[off])) <= 1e-3 * alpha + 1e-4
        assert np.max(np.abs(np.diag(r["G"]))) <= 1e-3
        assert np.all(np.abs(r["gb"]) <= 1e-4 * q + 1e-6)
        sums.append(np.abs(f["W"][off]).sum())
    assert sums[0] > sums[1] > sums[2]
