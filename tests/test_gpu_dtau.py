"""Derivative in tau (step a6) and the autograd binding, on the GPU against the FP64 oracle.

The oracle's dL/dtau is pinned to central finite differences of its own L (test_oracle_pins).  Here the GPU
value must match it within 1e-4 of sum_i |row contribution| (the scale of the terms that cancel in the
total), and the autograd gradients must match the oracle's dL/dW, dL/db and dL/dtau, and central finite
differences of the oracle L on sampled W entries (h = 1e-4)."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


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


def workload(n, T, seed):
    return synth.make_workload(None, n=n, n_exc=int(0.8 * n), p=0.1, w_exc=0.3, w_inh=1.2, w_self=-3.0, rate=8.0,
                               tau=0.01, dt=0.001, n_bins=T, seed=seed)


def params(w, seed):
    rng = np.random.default_rng(seed)
    n = w["n"]
    W = (w["W_true"] + rng.normal(0, 0.05, (n, n))).astype(np.float32)
    b = (w["b_true"] + rng.normal(0, 0.1, n)).astype(np.float32)
    return W, b


@pytest.mark.parametrize("prec", ["bf16", "f16"])
@pytest.mark.parametrize("n,T,seed", [(50, 20000, 0), (130, 5000, 2), (300, 70000, 4)])
def test_dtau_matches_oracle(ctx, prec, n, T, seed):
    w = workload(n, T, seed)
    W, b = params(w, seed + 1)
    ctx.set_problem(w["offs"], w["bins"], T, w["dt"], w["tau"], prec=prec)
    r = ctx.loglik_grad(torch.from_numpy(W).cuda(), torch.from_numpy(b).cuda(), tau_grad=True)
    ref = oracle.loglik_grad(w["offs"], w["bins"], T, w["dt"], w["tau"], W.astype(np.float64), b.astype(np.float64))
    scale = np.abs(ref["gtau_rows"]).sum()
    print(f"{prec} n={n} T={T}: dL/dtau gpu {r['gtau']:.6e} oracle {ref['gtau']:.6e} scale {scale:.3e}")
    assert abs(r["gtau"] - ref["gtau"]) <= 1e-4 * scale
    # a second request reuses the prepared spike part
    r2 = ctx.loglik_grad(torch.from_numpy(W).cuda(), torch.from_numpy(b).cuda(), tau_grad=True)
    assert r2["gtau"] == r["gtau"]


def test_dtau_after_new_tau(ctx):
    w = workload(50, 20000, 0)
    W, b = params(w, 3)
    ctx.set_problem(w["offs"], w["bins"], 20000, w["dt"], w["tau"], prec="bf16")
    ctx.loglik_grad(torch.from_numpy(W).cuda(), torch.from_numpy(b).cuda(), tau_grad=True)
    tau2 = 0.015
    ctx.prepare(tau2)  # the tau-dependent caches (and the spike part of dL/dtau) are recomputed
    r = ctx.loglik_grad(torch.from_numpy(W).cuda(), torch.from_numpy(b).cuda(), tau_grad=True)
    ref = oracle.loglik_grad(w["offs"], w["bins"], 20000, w["dt"], tau2, W.astype(np.float64), b.astype(np.float64))
    assert abs(r["gtau"] - ref["gtau"]) <= 1e-4 * np.abs(ref["gtau_rows"]).sum()
    assert r["L_total"] == pytest.approx(ref["L_total"], rel=1e-6)


def test_autograd_function(ctx, glm):
    from paper_1502_04993_gb300.autograd import glm_loglik
    w = workload(40, 12000, 5)
    W, b = params(w, 6)
    ctx.set_problem(w["offs"], w["bins"], 12000, w["dt"], w["tau"], prec="f16")
    Wt = torch.from_numpy(W).cuda().requires_grad_(True)
    bt = torch.from_numpy(b).cuda().requires_grad_(True)
    tau = torch.tensor(w["tau"], dtype=torch.float64, requires_grad=True)
    L = glm_loglik(ctx, Wt, bt, tau)
    (2.0 * L).backward()
    ref = oracle.loglik_grad(w["offs"], w["bins"], 12000, w["dt"], w["tau"], W.astype(np.float64), b.astype(np.float64))
    assert L.item() == pytest.approx(ref["L_total"], rel=1e-6)
    C, _ = ctx.spike_term()
    Cn = C.cpu().numpy()
    mag = Cn + (Cn - ref["G"])
    gW = Wt.grad.cpu().numpy().astype(np.float64) / 2.0
    assert np.max(np.abs(gW - ref["G"]) / (mag + 1e-300)) <= 2e-3
    q = np.diff(w["offs"]).astype(np.float64)
    assert np.all(np.abs(bt.grad.cpu().numpy() / 2.0 - ref["gb"]) <= 1e-5 * (q + np.abs(q - ref["gb"])) + 1e-6)
    assert tau.grad.item() / 2.0 == pytest.approx(ref["gtau"], abs=1e-4 * np.abs(ref["gtau_rows"]).sum())
    # central finite differences of the oracle L on sampled W entries (h = 1e-4)
    rng = np.random.default_rng(7)
    h = 1e-4
    for _ in range(8):
        i, j = rng.integers(0, 40, 2)
        Wp, Wm = W.astype(np.float64), W.astype(np.float64)
        Wp = Wp.copy()
        Wm = Wm.copy()
        Wp[i, j] += h
        Wm[i, j] -= h
        fd = (oracle.eval_rows(w["offs"], w["bins"], 12000, w["dt"], w["tau"], Wp, b.astype(np.float64), [i],
                               grad=False)["L"][0]
              - oracle.eval_rows(w["offs"], w["bins"], 12000, w["dt"], w["tau"], Wm, b.astype(np.float64), [i],
                                 grad=False)["L"][0]) / (2 * h)
        assert gW[i, j] == pytest.approx(fd, abs=2e-3 * mag[i, j] + 1e-6)
