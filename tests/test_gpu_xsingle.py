"""One 16-bit X (glm_set_x_split(ctx, 0)): the U product W_hi X + W_lo X, the spike term S X^T and the
gradient product E X^T all over the round-to-nearest 16-bit X, with no X_lo array and no X_lo products.

Tolerances.  FP16 keeps 11 significant bits of X.  Evaluated in FP64 with only X so rounded, L at the
N = 1000, 200 000-bin balanced network moves by 2.1e-7 of its size, rows by at most 6.7e-6 of
|L_i| + q_i and the gradient by 5e-5 in the componentwise measure: the 16-bit bounds (total 1e-6, rows
3e-5, gradient 2e-3) hold with room.  BF16 keeps 8 bits; the same evaluation moves L by 6.3e-6 and rows
by 5.3e-5, beyond those bounds, so BF16 with one X is checked against bounds that its rounding allows
(total 3e-5, rows 3e-4): it is the form the split X exists to improve on.  The spike term is compared
element by element with the oracle's: each of its q_i terms X_j[t] >= 0 is the FP32 scan's value (within
1e-7 of X) rounded to nearest in the 16-bit type (relative error at most u = 2^-11 for FP16, 2^-8 for
BF16; below the normal range at most half the subnormal spacing), and the tensor cores accumulate the sum
in FP32 (relative error below q_i 2^-23 even if each addition truncates), so
|C - C_exact| <= (u + 1e-7 + q_i 2^-23) C_exact + q_i 2^-25 (FP16) or q_i 2^-134 (BF16)."""
import numpy as np
import pytest
import torch

import oracle
import oracle.delays as od
import synth

pytestmark = pytest.mark.gpu

TOL = {"f16": dict(total=1e-6, row=3e-5, grad=2e-3), "bf16": dict(total=3e-5, row=3e-4, grad=2e-3)}
TDT = {"f16": torch.float16, "bf16": torch.bfloat16}


@pytest.fixture(scope="module")
def glm():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1502_04993_gb300 as g
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return g


def workload(n, T, seed):
    return synth.make_workload(None, n=n, n_exc=max(1, int(0.8 * n)), p=0.1, w_exc=0.3, w_inh=1.2, w_self=-3.0,
                               rate=8.0, tau=0.010, dt=0.001, n_bins=T, seed=seed)


def params(w, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    n = w["n"]
    W = (scale * w["W_true"] + rng.normal(0, 0.05, (n, n))).astype(np.float32)
    b = (w["b_true"] + rng.normal(0, 0.1, n)).astype(np.float32)
    return W, b


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def single(glm, w, prec, T=None, tau=None):
    c = glm.GLM(0)
    c.set_x_split(False)
    c.set_problem(w["offs"], w["bins"], T or w["n_bins"], w["dt"], tau or w["tau"], prec=prec)
    return c


def componentwise(G, G_ref, C):
    return float(np.max(np.abs(G - G_ref) / (C + (C - G_ref) + 1e-300)))


@pytest.mark.parametrize("prec", ["f16", "bf16"])
@pytest.mark.parametrize("n,T,seed,scale", [(50, 20000, 0, 1.0), (37, 9001, 1, 0.5), (130, 5000, 2, 1.0),
                                            (300, 70000, 3, 1.0)])
def test_single_x_matches_oracle(glm, prec, n, T, seed, scale):
    """Ragged N and T, more tiles than SMs; L, every row, the gradient, g_b and the spike term."""
    tol = TOL[prec]
    w = workload(n, T, seed)
    W, b = params(w, seed + 100, scale)
    with single(glm, w, prec) as c:
        r = c.loglik_grad(dev(W), dev(b))
        C = c.spike_term()[0].cpu().numpy()
    ref = oracle.loglik_grad(w["offs"], w["bins"], T, w["dt"], w["tau"], W.astype(np.float64), b.astype(np.float64))
    q = np.diff(w["offs"]).astype(np.float64)
    rel_tot = abs(r["L_total"] - ref["L_total"]) / abs(ref["L_total"])
    rel_rows = np.max(np.abs(r["L_rows"].cpu().numpy() - ref["L"]) / (np.abs(ref["L"]) + q))
    g = componentwise(r["G"].cpu().numpy(), ref["G"], C)
    X = oracle.filter(w["offs"], w["bins"], T, w["dt"], w["tau"])
    Cx = np.stack([X[:, w["bins"][w["offs"][i]:w["offs"][i + 1]]].sum(axis=1) for i in range(n)])
    u, sub = (2.0 ** -11, 2.0 ** -25) if prec == "f16" else (2.0 ** -8, 2.0 ** -134)
    bound = (u + 1e-7 + q[:, None] * 2.0 ** -23) * Cx + q[:, None] * sub
    c_err = float(np.max(np.abs(C - Cx) / (Cx + 1e-300)))
    print(f"{prec} single X n={n} T={T}: L total {rel_tot:.2e}, rows {rel_rows:.2e}, grad {g:.2e}, C vs exact {c_err:.2e}")
    assert rel_tot <= tol["total"] and rel_rows <= tol["row"] and g <= tol["grad"]
    assert np.all(np.abs(r["gb"].cpu().numpy() - ref["gb"]) <= tol["row"] * (q + np.abs(q - ref["gb"])) + 1e-9)
    assert np.all(np.abs(C - Cx) <= bound)


def test_single_x_differs_from_split_by_the_rounding(glm):
    """The option takes effect: the split and single forms of one problem differ, by about the rounding of X."""
    w = workload(130, 20000, 5)
    W, b = params(w, 6)
    with glm.GLM(0) as a, single(glm, w, "f16") as s:
        a.set_problem(w["offs"], w["bins"], w["n_bins"], w["dt"], w["tau"], prec="f16")
        La = a.loglik_grad(dev(W), dev(b), grad=False)["L_total"]
        Ls = s.loglik_grad(dev(W), dev(b), grad=False)["L_total"]
    d = abs(La - Ls) / abs(La)
    print(f"split vs single X: {d:.2e}")
    assert 0 < d <= 2e-6


@pytest.mark.parametrize("n,T,chunk", [(130, 70000, 16384), (37, 9001, 2048)])
def test_single_x_chunked_matches_stored(glm, n, T, chunk):
    w = workload(n, T, 3)
    W, b = params(w, 4)
    with single(glm, w, "f16") as a, glm.GLM(0) as c:
        c.set_x_split(False)
        c.set_chunk_bins(chunk)
        c.set_problem(w["offs"], w["bins"], T, w["dt"], w["tau"], prec="f16")
        ra = a.loglik_grad(dev(W), dev(b), tau_grad=True)
        rc = c.loglik_grad(dev(W), dev(b), tau_grad=True)
        Ca = a.spike_term()[0].cpu().numpy()
        La, Lc = ra["L_rows"].cpu().numpy(), rc["L_rows"].cpu().numpy()
        q = np.diff(w["offs"]).astype(np.float64)
        assert np.all(np.abs(La - Lc) <= 1e-12 * (np.abs(La) + q))
        assert rc["gtau"] == pytest.approx(ra["gtau"], rel=1e-12, abs=1e-9)
        assert np.max(np.abs(ra["G"].cpu().numpy() - rc["G"].cpu().numpy()) / (np.abs(Ca) + 1e-9)) <= 1e-5


@pytest.mark.parametrize("n,T,seed", [(50, 20000, 0), (130, 30000, 2)])
def test_single_x_dtau_matches_oracle(glm, n, T, seed):
    w = workload(n, T, seed)
    W, b = params(w, seed + 1)
    with single(glm, w, "f16") as c:
        r = c.loglik_grad(dev(W), dev(b), tau_grad=True)
    ref = oracle.loglik_grad(w["offs"], w["bins"], T, w["dt"], w["tau"], W.astype(np.float64), b.astype(np.float64))
    scale = np.abs(ref["gtau_rows"]).sum()
    print(f"single X dL/dtau {r['gtau']:.6e} oracle {ref['gtau']:.6e} scale {scale:.3e}")
    assert abs(r["gtau"] - ref["gtau"]) <= 1e-4 * scale


def test_single_x_fit_matches_oracle_fit(glm):
    """The plain workload (N = 50, 20 000 bins): the fit reaches the oracle's optimum to within the single
    X's objective offset, with identical labels."""
    w = synth.make_workload("glm_n50_t20k")
    fo = oracle.fit(w["offs"], w["bins"], w["n_bins"], w["dt"], w["tau"], eta=1e-10, max_iter=500)
    with single(glm, w, "f16") as c:
        r = c.fit(eta=1e-10, max_iter=500)
        assert r["rc"] >= 0 and r["report"]["maxiter"] == 0
        Wg = r["W"].cpu().numpy().astype(np.float64)
        bg = r["b"].cpu().numpy().astype(np.float64)
    args = (w["offs"], w["bins"], w["n_bins"], w["dt"], w["tau"])
    Lg = oracle.loglik_grad(*args, Wg, bg)["L_total"]
    Lo = oracle.loglik_grad(*args, fo["W"], fo["b"])["L_total"]
    print(f"single X fit: oracle L at the GPU fit {Lg:.9f}, at its own {Lo:.9f}; max |dW| {np.abs(Wg - fo['W']).max():.2e}")
    assert Lg <= Lo + 1e-9 * abs(Lo) and Lo - Lg <= 2e-6 * abs(Lo)
    lg, _ = glm.classify(Wg, "kmeans")
    lo, _ = glm.classify(fo["W"], "kmeans")
    assert np.array_equal(lg, lo)


def test_single_x_batch_matches_oracle(glm):
    ws = [synth.make_workload("glm_n50_t20k")]
    for n, T, seed in [(37, 9001, 1), (130, 12000, 2)]:
        ws.append(workload(n, T, seed))
    ctxs = [single(glm, w, "f16") for w in ws]
    try:
        res, rc = glm.fit_batch(ctxs, eta=1e-10, max_iter=500)
        assert rc >= 0
        for w, r in zip(ws, res):
            assert r["report"]["maxiter"] == 0 and r["report"]["stalled"] == 0
            args = (w["offs"], w["bins"], w["n_bins"], w["dt"], w["tau"])
            fo = oracle.fit(*args, eta=1e-10, max_iter=500)
            Lb = oracle.loglik_grad(*args, r["W"].cpu().numpy().astype(np.float64),
                                    r["b"].cpu().numpy().astype(np.float64))["L_total"]
            Lo = oracle.loglik_grad(*args, fo["W"], fo["b"])["L_total"]
            print(f"single X batch n={w['n']}: L oracle opt {Lo:.9f} batch {Lb:.9f}")
            assert Lb <= Lo + 1e-9 * abs(Lo) and Lo - Lb <= 2e-6 * abs(Lo)
    finally:
        for c in ctxs:
            c.close()


def test_single_x_row_classes_with_self_delay(glm):
    """Row classes with their own tau, source delay and self-delay (Sec. 2.4, Sec. 3.1) over the single X,
    against oracle.delays: every row of every class within the per-row bound, the gradient componentwise,
    and the network's L (the sum over the classes) within the total bound.  A class's own total is a sum of
    as few as 20 rows, whose X-rounding errors (up to ~1e-5 of a row) do not average out as over the
    network, so it is held to the per-row bound summed over its rows."""
    classes = [(0, 50, 0.010, 2, 1), (50, 100, 0.012, 4, 1), (100, 120, 0.010, 3, 3)]
    w = workload(120, 30000, 23)
    n = w["n"]
    W, b = params(w, 4)
    taus, ds, ss = np.zeros(n), np.zeros(n, dtype=np.int64), np.zeros(n, dtype=np.int64)
    for r0, r1, tau, d, s in classes:
        taus[r0:r1], ds[r0:r1], ss[r0:r1] = tau, d, s
    ref = od.loglik_grad_classes(w["offs"], w["bins"], w["n_bins"], w["dt"], taus, ds, W.astype(np.float64),
                                 b.astype(np.float64), self_delay_rows=ss)
    q = np.diff(w["offs"]).astype(np.float64)
    tol = TOL["f16"]
    L_net = 0.0
    for r0, r1, tau, d, s in classes:
        with glm.GLM(0) as c:
            c.set_x_split(False)
            c.set_source_delay(d)
            c.set_self_delay(s)
            c.set_problem(w["offs"], w["bins"], w["n_bins"], w["dt"], tau, prec="f16")
            c.set_row_range(r0, r1)
            r = c.loglik_grad(dev(W), dev(b))
            C = c.spike_term()[0].cpu().numpy()
        sl = slice(r0, r1)
        Lr, G = r["L_rows"].cpu().numpy(), r["G"].cpu().numpy()
        rel_tot = abs(r["L_total"] - ref["L"][sl].sum()) / abs(ref["L"][sl].sum())
        rel_rows = np.max(np.abs(Lr[sl] - ref["L"][sl]) / (np.abs(ref["L"][sl]) + q[sl]))
        g = componentwise(G[sl], ref["G"][sl], C[sl])
        print(f"single X class d={d} d_s={s}: L {rel_tot:.2e}, rows {rel_rows:.2e}, grad {g:.2e}")
        assert rel_rows <= tol["row"] and g <= tol["grad"]
        assert abs(r["L_total"] - ref["L"][sl].sum()) <= tol["row"] * (np.abs(ref["L"][sl]) + q[sl]).sum()
        L_net += r["L_total"]
    rel_net = abs(L_net - ref["L"].sum()) / abs(ref["L"].sum())
    print(f"single X classes: network L {rel_net:.2e}")
    assert rel_net <= tol["total"]
