"""X recomputed chunk by chunk (glm_set_chunk_bins): the same evaluation as with X stored.  Each U-product
tile sees the same operands in both forms, so L_i and dL/dtau agree to rounding of the final sums; E X^T is
summed over chunks in another order, so G agrees to FP32 rounding of its partial sums.  Both are checked
against the oracle, and a chunked fit against the oracle's fit."""
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


def workload(n, T, seed):
    return synth.make_workload(None, n=n, n_exc=int(0.8 * n), p=0.1, w_exc=0.3, w_inh=1.2, w_self=-3.0, rate=8.0,
                               tau=0.01, dt=0.001, n_bins=T, seed=seed)


@pytest.mark.parametrize("prec", ["bf16", "f16"])
@pytest.mark.parametrize("n,T,chunk", [(130, 70000, 16384), (37, 9001, 2048)])
def test_chunked_matches_stored(glm, prec, n, T, chunk):
    w = workload(n, T, 3)
    rng = np.random.default_rng(4)
    W = torch.from_numpy((w["W_true"] + rng.normal(0, 0.05, (n, n))).astype(np.float32)).cuda()
    b = torch.from_numpy((w["b_true"] + rng.normal(0, 0.1, n)).astype(np.float32)).cuda()
    with glm.GLM(0) as a, glm.GLM(0) as c:
        a.set_problem(w["offs"], w["bins"], T, w["dt"], w["tau"], prec=prec)
        c.set_chunk_bins(chunk)
        c.set_problem(w["offs"], w["bins"], T, w["dt"], w["tau"], prec=prec)
        ra = a.loglik_grad(W, b, tau_grad=True)
        rc = c.loglik_grad(W, b, tau_grad=True)
        La, Lc = ra["L_rows"].cpu().numpy(), rc["L_rows"].cpu().numpy()
        q = np.diff(w["offs"]).astype(np.float64)
        assert np.all(np.abs(La - Lc) <= 1e-12 * (np.abs(La) + q))
        assert rc["gtau"] == pytest.approx(ra["gtau"], rel=1e-12, abs=1e-9)
        Ga, Gc = ra["G"].cpu().numpy(), rc["G"].cpu().numpy()
        Ca, _ = a.spike_term()
        Cc, _ = c.spike_term()
        Ca, Cc = Ca.cpu().numpy(), Cc.cpu().numpy()
        assert np.max(np.abs(Ca - Cc) / (np.abs(Ca) + 1e-9)) <= 1e-6
        assert np.max(np.abs(Ga - Gc) / (np.abs(Ca) + 1e-9)) <= 1e-5
        ref = oracle.loglik_grad(w["offs"], w["bins"], T, w["dt"], w["tau"], W.cpu().numpy().astype(np.float64),
                                 b.cpu().numpy().astype(np.float64))
        assert abs(rc["L_total"] - ref["L_total"]) <= 1e-6 * abs(ref["L_total"])
        assert abs(rc["gtau"] - ref["gtau"]) <= 1e-4 * np.abs(ref["gtau_rows"]).sum()


def test_chunked_fit_matches_oracle_fit(glm):
    w = synth.make_workload("glm_n50_t20k")
    fo = oracle.fit(w["offs"], w["bins"], w["n_bins"], w["dt"], w["tau"], eta=1e-10, max_iter=500)
    with glm.GLM(0) as c:
        c.set_chunk_bins(4096)
        c.set_problem(w["offs"], w["bins"], w["n_bins"], w["dt"], w["tau"], prec="bf16")
        r = c.fit(eta=1e-10, max_iter=500)
        assert r["rc"] >= 0 and r["report"]["maxiter"] == 0
        W = r["W"].cpu().numpy().astype(np.float64)
        assert np.abs(W - fo["W"]).max() <= 3e-2


@pytest.fixture(scope="module")
def synfire():
    return synth.make_workload("glm_n2000_synfire_t3600s")


def test_full_size_synfire_chunked_sampled_rows(glm, synfire):
    """N = 2000 with the synfire chain, 3.6M bins (one hour at 1 ms), X recomputed in chunks of 262144 bins,
    BF16, with dL/dtau requested: three sampled rows against the oracle, which
    streams over the bins at any size.  Tolerances as for the stored form: per row (|L_i| + q_i) x 3e-5,
    gradient 2e-3 in the measure against C_ij + (C_ij - G_ij); dL/dtau finite."""
    w = synfire
    n, T = w["n"], w["n_bins"]
    W = w["W_true"].astype(np.float32)
    b = w["b_true"].astype(np.float32)
    rows = np.array([0, n // 2 + 7, n - 1], dtype=np.int32)
    with glm.GLM(0) as c:
        c.set_chunk_bins(262144)
        c.set_problem(w["offs"], w["bins"], T, w["dt"], w["tau"], prec="bf16")
        r = c.loglik_grad(torch.from_numpy(W).cuda(), torch.from_numpy(b).cuda(), tau_grad=True)
        Cs, _ = c.spike_term()
        Cr = Cs.cpu().numpy()[rows]
    ref = oracle.eval_rows(w["offs"], w["bins"], T, w["dt"], w["tau"], W.astype(np.float64), b.astype(np.float64),
                           rows)
    q = np.diff(w["offs"])[rows].astype(np.float64)
    rel = np.abs(r["L_rows"].cpu().numpy()[rows] - ref["L"]) / (np.abs(ref["L"]) + q)
    Gr = r["G"].cpu().numpy()[rows]
    g = float(np.max(np.abs(Gr - ref["G"]) / (Cr + (Cr - ref["G"]) + 1e-300)))
    print(f"synfire chunked: rows {rows.tolist()} rel {rel}, grad {g:.2e}, dL/dtau {r['gtau']:.6e}")
    assert np.all(rel <= 3e-5) and g <= 2e-3
    assert np.isfinite(r["gtau"])


def test_full_size_synfire_finite_differences(glm, synfire):
    """The differentiation workload as specified: N = 2000 with the synfire chain, 3.6M bins, X recomputed in
    chunks of 262 144 bins, BF16, through the autograd Function, at W away from the generating weights.
      * dL/dW on 32 seeded random entries, one in each of 32 rows, against central differences (h = 1e-4) of
        the FP64 oracle's L_i (one oracle pass per sign: each row sees only its own perturbed entry), and the
        32 rows' whole gradient against the oracle's (componentwise measure, 2e-3); dL/db of those rows.
      * dL/dtau against central differences of the GPU's own L at tau (1 +- 1e-3): the difference quotient
        carries the evaluation's error of ~1e-8 |L| divided by the step, plus a truncation error of order
        (1e-3)^2, so the bound is 1e-8 |L| / h + 1e-3 |dL/dtau|."""
    from paper_1502_04993_gb300.autograd import glm_loglik
    w = synfire
    n, T = w["n"], w["n_bins"]
    rng = np.random.default_rng(21)
    W = (w["W_true"] + rng.normal(0, 0.02, (n, n))).astype(np.float32)
    b = w["b_true"].astype(np.float32)
    rows = np.sort(rng.choice(n, 32, replace=False)).astype(np.int32)
    cols = rng.integers(0, n, 32)
    with glm.GLM(0) as c:
        c.set_chunk_bins(262144)
        c.set_problem(w["offs"], w["bins"], T, w["dt"], w["tau"], prec="bf16")
        Wt = torch.from_numpy(W).cuda().requires_grad_(True)
        bt = torch.from_numpy(b).cuda().requires_grad_(True)
        tau = torch.tensor(w["tau"], dtype=torch.float64, requires_grad=True)
        L = glm_loglik(c, Wt, bt, tau)
        L.backward()
        gW = Wt.grad.cpu().numpy().astype(np.float64)
        gb = bt.grad.cpu().numpy().astype(np.float64)
        gtau = tau.grad.item()
        Cs = c.spike_term()[0].cpu().numpy()
        ht = 1e-3 * w["tau"]
        with torch.no_grad():
            Lp = glm_loglik(c, Wt, bt, w["tau"] + ht).item()
            Lm = glm_loglik(c, Wt, bt, w["tau"] - ht).item()
    args = (w["offs"], w["bins"], T, w["dt"], w["tau"])
    W64, b64 = W.astype(np.float64), b.astype(np.float64)
    ref = oracle.eval_rows(*args, W64, b64, rows)
    h = 1e-4
    Wp, Wm = W64.copy(), W64.copy()
    Wp[rows, cols] += h
    Wm[rows, cols] -= h
    fd = (oracle.eval_rows(*args, Wp, b64, rows, grad=False)["L"]
          - oracle.eval_rows(*args, Wm, b64, rows, grad=False)["L"]) / (2 * h)
    Cr = Cs[rows]
    mag = Cr + (Cr - ref["G"])
    g_rows = float(np.max(np.abs(gW[rows] - ref["G"]) / (mag + 1e-300)))
    fd_err = np.abs(gW[rows, cols] - fd) / (mag[np.arange(32), cols] + 1e-300)
    fd_vs_oracle = np.abs(ref["G"][np.arange(32), cols] - fd) / (mag[np.arange(32), cols] + 1e-300)
    q = np.diff(w["offs"])[rows].astype(np.float64)
    fd_tau = (Lp - Lm) / (2 * ht)
    print(f"config 3 FD: grad rows {g_rows:.2e}, GPU vs FD max {fd_err.max():.2e}, oracle vs FD max "
          f"{fd_vs_oracle.max():.2e}; dL/dtau {gtau:.6e} vs FD {fd_tau:.6e} (L {L.item():.6e})")
    assert g_rows <= 2e-3
    assert np.all(fd_vs_oracle <= 1e-6)   # the oracle's gradient is its own L's derivative (O(h^2) = 1e-8)
    assert np.all(fd_err <= 2e-3)
    assert np.all(np.abs(gb[rows] - ref["gb"]) <= 3e-5 * (q + np.abs(q - ref["gb"])) + 1e-9)
    assert abs(fd_tau - gtau) <= 1e-8 * abs(L.item()) / ht + 1e-3 * abs(gtau)
