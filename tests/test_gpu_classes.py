"""Per-neuron time constants and delays (glm_set_source_delay, glm_set_row_range, glm_fit_classes) on
the GPU against the FP64 oracle (oracle.delays): one context per class of rows with equal (tau, delay).

Tolerances as for the whole-network evaluations: 16-bit forms total relative 1e-6 (here over the class's
rows), per row (|L_i| + q_i) x 3e-5 (BF16), gradient 2e-3 in the componentwise measure against
C_ij + (C_ij - G_ij); the plain FP32 form per row 5e-8, gradient 1e-5 and class total 1e-9, the bound of a
whole network's total.  Rows outside a context's range come back as zeros."""
import numpy as np
import pytest
import torch

import synth
from oracle import delays as od

pytestmark = pytest.mark.gpu

CLASSES = [(0, 40, 0.008, 1), (40, 80, 0.012, 2), (80, 120, 0.010, 4)]  # rows [r0, r1), tau, delay in bins


@pytest.fixture(scope="module")
def glm():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1502_04993_gb300 as g
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return g


def workload(n=120, T=20000, seed=21):
    return synth.make_workload(None, n=n, n_exc=int(0.8 * n), p=0.1, w_exc=0.3, w_inh=1.2, w_self=-3.0, rate=8.0,
                               tau=0.010, dt=0.001, n_bins=T, seed=seed)


def row_params(n):
    taus, ds = np.zeros(n), np.zeros(n, dtype=np.int64)
    for r0, r1, tau, d in CLASSES:
        taus[r0:r1], ds[r0:r1] = tau, d
    return taus, ds


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def contexts(glm, w, prec):
    out = []
    for r0, r1, tau, d in CLASSES:
        c = glm.GLM(0)
        c.set_source_delay(d)
        c.set_problem(w["offs"], w["bins"], w["n_bins"], w["dt"], tau, prec=prec)
        c.set_row_range(r0, r1)
        out.append(c)
    return out


@pytest.mark.parametrize("prec,tol", [("bf16", dict(tot=1e-6, row=3e-5, grad=2e-3)),
                                      ("f32", dict(tot=1e-9, row=5e-8, grad=1e-5))])
def test_classes_match_oracle(glm, prec, tol):
    w = workload()
    n = w["n"]
    rng = np.random.default_rng(3)
    W = (w["W_true"] + rng.normal(0, 0.05, (n, n))).astype(np.float32)
    b = (w["b_true"] + rng.normal(0, 0.1, n)).astype(np.float32)
    taus, ds = row_params(n)
    ref = od.loglik_grad_classes(w["offs"], w["bins"], w["n_bins"], w["dt"], taus, ds, W.astype(np.float64),
                                 b.astype(np.float64))
    q = np.diff(w["offs"]).astype(np.float64)
    cs = contexts(glm, w, prec)
    try:
        for (r0, r1, tau, d), c in zip(CLASSES, cs):
            r = c.loglik_grad(to_dev(W), to_dev(b))
            C, _ = c.spike_term()
            Lr = r["L_rows"].cpu().numpy()
            G = r["G"].cpu().numpy()
            gb = r["gb"].cpu().numpy()
            sl = slice(r0, r1)
            tot_ref = ref["L"][sl].sum()
            rel_tot = abs(r["L_total"] - tot_ref) / abs(tot_ref)
            rel_rows = np.max(np.abs(Lr[sl] - ref["L"][sl]) / (np.abs(ref["L"][sl]) + q[sl]))
            Cr = C.cpu().numpy()[sl]
            g = np.max(np.abs(G[sl] - ref["G"][sl]) / (Cr + (Cr - ref["G"][sl]) + 1e-300))
            print(f"{prec} class tau={tau} d={d}: L rel {rel_tot:.2e}, rows {rel_rows:.2e}, grad {g:.2e}")
            assert rel_tot <= tol["tot"] and rel_rows <= tol["row"] and g <= tol["grad"]
            assert np.all(np.abs(gb[sl] - ref["gb"][sl]) <= tol["row"] * (q[sl] + np.abs(q[sl] - ref["gb"][sl])) + 1e-9)
            out = np.r_[0:r0, r1:n]
            assert np.all(Lr[out] == 0.0) and np.all(G[out] == 0.0) and np.all(gb[out] == 0.0)
    finally:
        for c in cs:
            c.close()


def test_fit_classes_reaches_the_oracle_optimum(glm):
    w = workload(T=60000, seed=22)
    n = w["n"]
    taus, ds = row_params(n)
    cs = contexts(glm, w, "bf16")
    try:
        res = glm.fit_classes(cs, eta=1e-10, max_iter=300)
    finally:
        for c in cs:
            c.close()
    W = res["W"].cpu().numpy().astype(np.float64)
    b = res["b"].cpu().numpy().astype(np.float64)
    ref = od.loglik_grad_classes(w["offs"], w["bins"], w["n_bins"], w["dt"], taus, ds, W, b)
    g = np.abs(ref["G"])
    q = np.diff(w["offs"]).astype(np.float64)
    print(f"fit classes: {res['report']}, max |G| {g.max():.3e}, max |gb|/q {np.max(np.abs(ref['gb']) / (q + 1)):.2e}")
    assert res["rc"] >= 0 and res["report"]["excluded"] == 0
    assert set(res["status"].tolist()) <= {0, 4}
    assert np.all(np.abs(ref["gb"]) <= 1e-2 * (q + 1))
    # at the optimum of each row the gradient vanishes up to the fit's stopping rule: compare with the
    # gradient at the generating weights of the grid model
    g0 = np.abs(od.loglik_grad_classes(w["offs"], w["bins"], w["n_bins"], w["dt"], taus, ds, w["W_true"],
                                       w["b_true"])["G"])
    assert np.median(g) <= 1e-2 * np.median(g0)


def test_row_range_and_delay_errors(glm):
    w = workload(n=16, T=3000, seed=5)
    with glm.GLM(0) as c:
        with pytest.raises(glm.GLMError):
            c.set_source_delay(0)
        with pytest.raises(glm.GLMError):
            c.set_row_range(0, 4)  # no problem yet
        c.set_problem(w["offs"], w["bins"], 3000, 0.001, 0.01, prec="bf16")
        for bad in [(-1, 4), (4, 4), (5, 17)]:
            with pytest.raises(glm.GLMError):
                c.set_row_range(*bad)
        c.set_row_range(0, 8)
        with pytest.raises(glm.GLMError):
            glm.fit_batch([c])
        c.set_row_range(0, 0)  # all rows again
        r = c.loglik_grad(to_dev(w["W_true"].astype(np.float32)), to_dev(w["b_true"].astype(np.float32)))
        assert np.all(r["L_rows"].cpu().numpy() != 0.0)


SELF_CLASSES = [(0, 50, 0.010, 2, 1), (50, 100, 0.012, 4, 1), (100, 120, 0.010, 3, 3)]  # + self-delay in bins


@pytest.mark.parametrize("prec,tol", [("bf16", dict(tot=1e-6, row=3e-5, grad=2e-3)),
                                      ("f16", dict(tot=1e-6, row=4e-6, grad=2e-3))])
def test_self_delay_matches_oracle(glm, prec, tol):
    """The paper's separate self-delay (Sec. 2.4, Sec. 3.1: d_s = one bin, d longer): each class's rows see
    their own train after d_s bins and every other train after d, against oracle.delays with the self-delay
    (pinned to the per-pair definition); the last class has d_s = d (no change)."""
    w = workload(T=30000, seed=23)
    n = w["n"]
    rng = np.random.default_rng(4)
    W = (w["W_true"] + rng.normal(0, 0.05, (n, n))).astype(np.float32)
    b = (w["b_true"] + rng.normal(0, 0.1, n)).astype(np.float32)
    taus, ds, ss = np.zeros(n), np.zeros(n, dtype=np.int64), np.zeros(n, dtype=np.int64)
    for r0, r1, tau, d, s in SELF_CLASSES:
        taus[r0:r1], ds[r0:r1], ss[r0:r1] = tau, d, s
    ref = od.loglik_grad_classes(w["offs"], w["bins"], w["n_bins"], w["dt"], taus, ds, W.astype(np.float64),
                                 b.astype(np.float64), self_delay_rows=ss)
    plain = od.loglik_grad_classes(w["offs"], w["bins"], w["n_bins"], w["dt"], taus, ds, W.astype(np.float64),
                                   b.astype(np.float64))
    q = np.diff(w["offs"]).astype(np.float64)
    cs = []
    try:
        for r0, r1, tau, d, s in SELF_CLASSES:
            c = glm.GLM(0)
            cs.append(c)
            c.set_source_delay(d)
            c.set_self_delay(s)
            c.set_problem(w["offs"], w["bins"], w["n_bins"], w["dt"], tau, prec=prec)
            c.set_row_range(r0, r1)
            r = c.loglik_grad(to_dev(W), to_dev(b))
            C = c.spike_term()[0].cpu().numpy()
            sl = slice(r0, r1)
            Lr, G = r["L_rows"].cpu().numpy(), r["G"].cpu().numpy()
            tot_ref = ref["L"][sl].sum()
            rel_tot = abs(r["L_total"] - tot_ref) / abs(tot_ref)
            rel_rows = np.max(np.abs(Lr[sl] - ref["L"][sl]) / (np.abs(ref["L"][sl]) + q[sl]))
            Cr = C[sl]
            g = np.max(np.abs(G[sl] - ref["G"][sl]) / (Cr + (Cr - ref["G"][sl]) + 1e-300))
            moved = np.max(np.abs(plain["L"][sl] - ref["L"][sl]) / (np.abs(ref["L"][sl]) + q[sl]))
            print(f"{prec} class d={d} d_s={s}: L rel {rel_tot:.2e}, rows {rel_rows:.2e}, grad {g:.2e} "
                  f"(the self-delay moves L_i by {moved:.2e})")
            assert rel_tot <= tol["tot"] and rel_rows <= tol["row"] and g <= tol["grad"]
            gb = r["gb"].cpu().numpy()
            assert np.all(np.abs(gb[sl] - ref["gb"][sl]) <= tol["row"] * (q[sl] + np.abs(q[sl] - ref["gb"][sl])) + 1e-9)
            if s < d:
                assert moved > 100 * tol["row"]  # the check would see a missing self-delay
    finally:
        for c in cs:
            c.close()


def test_self_delay_fit_and_errors(glm):
    """A fit with the self-delay reaches its optimum (the oracle's gradient with the self-delay vanishes there up
    to the stopping rule), and the combinations the self-delay does not serve are refused."""
    w = workload(n=60, T=40000, seed=24)
    n = w["n"]
    with glm.GLM(0) as c:
        c.set_source_delay(3)
        c.set_self_delay(1)
        c.set_problem(w["offs"], w["bins"], w["n_bins"], w["dt"], w["tau"], prec="bf16")
        r = c.fit(eta=1e-10, max_iter=300)
        assert r["rc"] >= 0
        W = r["W"].cpu().numpy().astype(np.float64)
        b = r["b"].cpu().numpy().astype(np.float64)
        ref = od.loglik_grad_classes(w["offs"], w["bins"], w["n_bins"], w["dt"], [w["tau"]] * n, [3] * n, W, b,
                                     self_delay_rows=[1] * n)
        g0 = od.loglik_grad_classes(w["offs"], w["bins"], w["n_bins"], w["dt"], [w["tau"]] * n, [3] * n,
                                    w["W_true"], w["b_true"], self_delay_rows=[1] * n)["G"]
        print(f"self-delay fit: {r['report']}, median |G| {np.median(np.abs(ref['G'])):.2e} vs "
              f"{np.median(np.abs(g0)):.2e} at the generating weights")
        assert np.median(np.abs(ref["G"])) <= 1e-2 * np.median(np.abs(g0))
        with pytest.raises(glm.GLMError) as e:
            c.loglik_grad(to_dev(W.astype(np.float32)), to_dev(b.astype(np.float32)), tau_grad=True)
        assert e.value.code == -10
        with pytest.raises(glm.GLMError) as e:
            c.set_problem(w["offs"], w["bins"], w["n_bins"], w["dt"], w["tau"], prec="f32")
        assert e.value.code == -10
        c.set_chunk_bins(8192)
        with pytest.raises(glm.GLMError) as e:
            c.set_problem(w["offs"], w["bins"], w["n_bins"], w["dt"], w["tau"], prec="bf16")
        assert e.value.code == -10
        with pytest.raises(glm.GLMError):
            c.set_self_delay(-1)
