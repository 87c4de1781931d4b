"""glm_fit on the GPU against the FP64 oracle's fit, and recovery of a known directed network.

The optimum of each row is unique (concave problem, App. A), so the GPU and the oracle must land on the
same W, b up to the stopping tolerance: with eta = 1e-10 on L_i the residual parameter error is about
sqrt(2 eta |L_i| / curvature), a few 1e-4 on the N = 50 workload.  The BF16 path evaluates L with relative
error ~1e-6, so its line search stalls a little earlier near the optimum; its bound is looser.
Classification labels from the two fits agree except for weights closer to a decision boundary than the
W difference (the reading of ties in the classification)."""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from oracle.classify import truth_labels

pytestmark = pytest.mark.gpu

CHAIN_W = np.array([[-2.0, 0.0, 0.0, 0.0],
                    [1.0, -2.0, 0.0, 0.0],
                    [0.0, -1.0, -2.0, 0.0],
                    [0.0, 0.0, 0.8, -2.0]])


@pytest.fixture(scope="module")
def glm():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1502_04993_gb300 as g
    return g


@pytest.fixture(scope="module")
def ctx(glm):
    c = glm.GLM(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def small():
    w = synth.make_workload("glm_n50_t20k")
    f = oracle.fit(w["offs"], w["bins"], w["n_bins"], w["dt"], w["tau"], eta=1e-10, max_iter=500)
    return w, f


@pytest.mark.parametrize("prec,wtol", [("f32", 5e-3), ("bf16", 3e-2), ("f16", 3e-2)])
def test_fit_matches_oracle_fit(ctx, glm, small, prec, wtol):
    w, fo = small
    ctx.set_problem(w["offs"], w["bins"], w["n_bins"], w["dt"], w["tau"], prec=prec)
    r = ctx.fit(eta=1e-10, max_iter=500)
    rep = r["report"]
    print(f"{prec}: {rep}")
    assert r["rc"] >= 0
    assert rep["maxiter"] == 0
    W = r["W"].cpu().numpy().astype(np.float64)
    b = r["b"].cpu().numpy().astype(np.float64)
    dW = np.abs(W - fo["W"])
    print(f"{prec}: max |dW| {dW.max():.2e}, max |db| {np.abs(b - fo['b']).max():.2e}")
    assert dW.max() <= wtol
    assert np.abs(b - fo["b"]).max() <= wtol
    # classification of the two fits: identical except within the W difference of a decision boundary
    lab_g, _ = oracle.classify(W, "kmeans")
    lab_o, model = oracle.classify(fo["W"], "kmeans")
    c = model["centroids"]
    bounds = np.array([(c[0] + c[1]) / 2, (c[1] + c[2]) / 2])
    near = np.min(np.abs(fo["W"][..., None] - bounds), axis=-1) < 10 * dW.max()
    assert np.all((lab_g == lab_o) | near)


def test_fit_gradient_vanishes_and_bias_stationary(ctx, small):
    """At the returned point the oracle's gradient is ~0 and q_i = dt sum_t e^{U_i} (Sec. 2.3.3)."""
    w, _ = small
    ctx.set_problem(w["offs"], w["bins"], w["n_bins"], w["dt"], w["tau"], prec="f32")
    r = ctx.fit(eta=1e-12, max_iter=800)
    W = r["W"].cpu().numpy().astype(np.float64)
    b = r["b"].cpu().numpy().astype(np.float64)
    ref = oracle.loglik_grad(w["offs"], w["bins"], w["n_bins"], w["dt"], w["tau"], W, b)
    q = np.diff(w["offs"]).astype(np.float64)
    assert np.all(np.abs(ref["gb"]) <= 1e-3 * q)
    assert np.abs(ref["G"]).max() <= 1e-2


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_fit_recovers_directed_chain(ctx, prec):
    n, T, dt, tau = 4, 200_000, 1e-3, 1e-2
    offs, bins = synth.simulate(CHAIN_W, np.full(n, math.log(20.0)), tau, dt, T, seed=21)
    ctx.set_problem(offs, bins, T, dt, tau, prec=prec)
    r = ctx.fit(eta=1e-12, max_iter=300)
    W = r["W"].cpu().numpy()
    assert np.abs(W - CHAIN_W).max() < 0.15, W


def test_fit_degenerate_row_and_ga(ctx):
    n, T, dt, tau = 3, 20_000, 1e-3, 1e-2
    W0 = np.array([[-1.0, 0.0, 0.0], [0.8, -1.0, 0.0], [0.0, 0.0, -1.0]])
    offs, bins = synth.simulate(W0, np.full(n, math.log(15.0)), tau, dt, T, seed=5)
    offs4 = np.concatenate([offs, [offs[-1]]]).astype(np.int64)  # a silent fourth neuron
    ctx.set_problem(offs4, bins, T, dt, tau, prec="f32")
    r1 = ctx.fit(method="lbfgs", eta=1e-13, max_iter=500)
    r2 = ctx.fit(method="ga", eta=1e-13, max_iter=5000)
    assert r1["status"][3] == 3
    assert r1["b"][3].item() == pytest.approx(math.log(1e-3), rel=1e-6)
    assert torch.all(r1["W"][3] == 0)
    fo = oracle.fit(offs4, bins, T, dt, tau, eta=1e-13, max_iter=500)
    assert np.allclose(r1["W"].cpu().numpy()[:3], fo["W"][:3], atol=2e-3)
    assert np.allclose(r2["W"].cpu().numpy()[:3], fo["W"][:3], atol=5e-3)
    assert r1["report"]["iterations"] < r2["report"]["iterations"]


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_fit_short_recording_stays_finite(ctx, prec):
    """Far fewer spikes per row than parameters: some weights have no finite maximum and run off while b_i
    falls far below U.  e^(U - b) then passes the FP32 range although e^U does not; the fit must still
    return finite parameters and a finite log-likelihood rather than an overflow error."""
    w = synth.make_workload(None, n=200, n_exc=160, p=0.1, w_exc=0.2, w_inh=0.8, w_self=-6.25, rate=8.0,
                            tau=0.01, dt=0.001, n_bins=6000, seed=9)
    ctx.set_problem(w["offs"], w["bins"], w["n_bins"], w["dt"], w["tau"], prec=prec)
    r = ctx.fit(eta=1e-9, max_iter=300)
    assert r["rc"] >= 0
    assert torch.isfinite(r["W"]).all() and torch.isfinite(r["b"]).all()
    assert math.isfinite(r["report"]["L"])


@pytest.mark.parametrize("prec,wtol", [("f32", 5e-3), ("bf16", 3e-2)])
def test_l1_penalised_fit_matches_oracle(ctx, prec, wtol):
    """Sec. 2.5: the smooth l1 MAP fit (Eq. 16-17) against the oracle's; at the GPU's point the oracle's own
    gradient balances the penalty, alpha W / sqrt(W^2 + eps), off the diagonal."""
    w = synth.make_workload("glm_n50_t20k", n_bins=8000)
    alpha, eps = 2.0, 1e-4
    fo = oracle.fit(w["offs"], w["bins"], 8000, w["dt"], w["tau"], eta=1e-12, max_iter=1000, alpha=alpha, eps=eps)
    ctx.set_problem(w["offs"], w["bins"], 8000, w["dt"], w["tau"], prec=prec)
    r = ctx.fit(eta=1e-12, max_iter=1000, alpha=alpha, eps=eps)
    assert r["rc"] >= 0 and r["report"]["maxiter"] == 0
    W = r["W"].cpu().numpy().astype(np.float64)
    b = r["b"].cpu().numpy().astype(np.float64)
    assert np.abs(W - fo["W"]).max() <= wtol
    g = oracle.loglik_grad(w["offs"], w["bins"], 8000, w["dt"], w["tau"], W, b)
    off = ~np.eye(W.shape[0], dtype=bool)
    resid = (g["G"] - alpha * W / np.sqrt(W ** 2 + eps))[off]
    scale = np.abs(g["G"]).max() + alpha
    assert np.abs(resid).max() <= (2e-3 if prec == "f32" else 5e-2) * scale


def test_cross_validation_recovers_tau(glm):
    """Sec. 3.2 / 2.5: fit on the first 60 % of a recording, score on the rest, over a grid of tau and alpha.
    The data were generated with tau = 10 ms, which must win; every grid value must equal the oracle's
    validation log-likelihood at the GPU fit."""
    w = synth.make_workload("glm_n50_t20k")
    (tr, va) = glm.split_recording(w["offs"], w["bins"], w["n_bins"], 12000)
    taus = [0.005, 0.01, 0.02]
    alphas = [0.0, 0.5, 2.0]
    with glm.GLM(0) as a, glm.GLM(0) as v:
        a.set_problem(tr[0], tr[1], tr[2], w["dt"], w["tau"], prec="bf16")
        v.set_problem(va[0], va[1], va[2], w["dt"], w["tau"], prec="bf16")
        res = glm.cross_validate(a, v, alphas, taus, eta=1e-10, max_iter=500)
        L = res["L_valid"]
        print(L)
        kt, ka = res["best"]
        assert taus[kt] == 0.01
        assert L[kt, ka] == L.max()
        Lo = oracle.loglik_grad(va[0], va[1], va[2], w["dt"], taus[kt], res["W"].cpu().numpy().astype(np.float64),
                                res["b"].cpu().numpy().astype(np.float64))["L_total"]
        assert abs(L[kt, ka] - Lo) <= 1e-6 * abs(Lo)
