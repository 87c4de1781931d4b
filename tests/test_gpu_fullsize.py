"""Parity at the full N = 1000, 1.8M-bin size of the balanced-network workload (the benchmark's launch
configuration), against the FP64 oracle on the host cores:

  * the whole-network log-likelihood, every row of it (the oracle streams all 1000 rows, a few minutes on
    the host): total relative 1e-6 for BF16 and 1e-9 for the plain FP32 form, every row within its
    per-row bound, and the gradient on 32 seeded random rows (componentwise measure);
  * a seeded subset of 16 rows fitted by the oracle from W = 0 (rows are independent problems, Sec. 2.2,
    so a subset fit is exact) against the same rows of the GPU's fits of the whole network, in the plain
    FP32 form and in BF16.  The stopping rule of Sec. 2.6.3 bounds the relative gain of the last iteration
    (eta = 1e-10), not the distance to the optimum: on these rows either fit ends up to ~1e-8 of L_i short
    of it (the oracle's own fit lands 1.2e-8 below the FP32 GPU fit's point on one row, measured), so the
    oracle's L_i at the GPU's rows and at its own rows differ by at most 2e-8 either way for the FP32 form.
    For BF16 the GPU's fit may lie up to 2e-6 below: its objective differs from the exact one by the
    tensor cores' FP32 accumulation (the FP16 fit lands equally far, ~6e-7 of L, so the X_hi + X_lo
    rounding is not the cause; the MER is unchanged).  The labels of each fit agree with the
    oracle's under one classifier (the GMM fitted to the GPU's whole W), apart from entries in the band where
    the two fits' difference can move a weight across a decision boundary (|W - boundary| < 10 max|dW|),
    which are counted.

W is perturbed away from the generating weights (the optimum of the fit is not where these bounds are
easiest)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle.classify import gmm_assign

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def glm():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1502_04993_gb300 as g
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return g


@pytest.fixture(scope="module")
def full():
    w = synth.make_workload("glm_n1000_t1800s")
    rng = np.random.default_rng(11)
    n = w["n"]
    W = (w["W_true"] + rng.normal(0, 0.02, (n, n))).astype(np.float32)
    b = (w["b_true"] + rng.normal(0, 0.05, n)).astype(np.float32)
    return w, W, b


@pytest.fixture(scope="module")
def oracle_rows(full):
    """The oracle's L_i for every row (no gradient), and its gradient on 32 seeded random rows."""
    w, W, b = full
    n, T = w["n"], w["n_bins"]
    args = (w["offs"], w["bins"], T, w["dt"], w["tau"], W.astype(np.float64), b.astype(np.float64))
    allL = oracle.eval_rows(*args, grad=False)
    rows = np.sort(np.random.default_rng(12).choice(n, 32, replace=False)).astype(np.int32)
    g = oracle.eval_rows(*args, rows)
    return allL, g


def metric10(G, G_ref, C_ref):
    mag = C_ref + (C_ref - G_ref)
    return float(np.max(np.abs(G - G_ref) / (mag + 1e-300)))


@pytest.mark.parametrize("prec,tot,row,grad", [("bf16", 1e-6, 3e-5, 2e-3), ("f16x1", 1e-6, 3e-5, 2e-3),
                                               ("f32", 1e-9, 5e-8, 1e-5)])
def test_full_size_whole_network(glm, full, oracle_rows, prec, tot, row, grad):
    """f16x1: X held as one FP16 array (no X_lo), the benchmark's default form."""
    w, W, b = full
    allL, g = oracle_rows
    q = np.diff(w["offs"]).astype(np.float64)
    with glm.GLM(0) as c:
        c.set_x_split(not prec.endswith("x1"))
        c.set_problem(w["offs"], w["bins"], w["n_bins"], w["dt"], w["tau"], prec=prec.replace("x1", ""))
        r = c.loglik_grad(torch.from_numpy(W).cuda(), torch.from_numpy(b).cuda())
        C = c.spike_term()[0].cpu().numpy()
        Lr = r["L_rows"].cpu().numpy()
        G = r["G"].cpu().numpy()
    rel_tot = abs(r["L_total"] - allL["L_total"]) / abs(allL["L_total"])
    rel_rows = np.max(np.abs(Lr - allL["L"]) / (np.abs(allL["L"]) + q))
    ge = metric10(G[g["rows"]], g["G"], C[g["rows"]])
    print(f"{prec} N=1000 T=1.8M: L total rel {rel_tot:.2e}, rows max {rel_rows:.2e}, grad (32 rows) {ge:.2e}")
    assert rel_tot <= tot
    assert rel_rows <= row
    assert ge <= grad


@pytest.fixture(scope="module")
def oracle_subset_fit(full):
    w, _, _ = full
    rows = np.sort(np.random.default_rng(13).choice(w["n"], 16, replace=False)).astype(np.int32)
    fo = oracle.fit(w["offs"], w["bins"], w["n_bins"], w["dt"], w["tau"], eta=1e-10, max_iter=500, rows=rows)
    assert np.all(fo["status"] == oracle.FIT_CONVERGED)
    return rows, fo


@pytest.mark.parametrize("prec,gap_bound,gap_low", [("f32", 2e-8, -2e-8), ("bf16", 2e-6, -2e-8),
                                                     ("f16x1", 2e-6, -2e-8), ("f16x1+f32", 2e-8, -2e-8)])
def test_full_size_subset_fit_matches_oracle(glm, full, oracle_subset_fit, prec, gap_bound, gap_low):
    """"f16x1": FP16 with X as one array; "f16x1+f32": that fit finished by the FP32 form from its result
    (warm start), which removes the 16-bit objective's offset from the exact optimum."""
    w, _, _ = full
    n, T = w["n"], w["n_bins"]
    rows, fo = oracle_subset_fit
    with glm.GLM(0) as c:
        r = None
        for p in prec.split("+"):
            c.set_x_split(not p.endswith("x1"))
            c.set_problem(w["offs"], w["bins"], T, w["dt"], w["tau"], prec=p.replace("x1", ""))
            r = c.fit(r["W"], r["b"], eta=1e-10, max_iter=500) if r is not None else c.fit(eta=1e-10, max_iter=500)
            print(f"{p} fit: {r['report']['seconds']:.2f} s, {r['report']['iterations']} iterations, "
                  f"{r['report']['evaluations']} evaluations, {r['report']['at_floor']} rows at the floor")
        Wg = r["W"].cpu().numpy().astype(np.float64)
        bg = r["b"].cpu().numpy().astype(np.float64)
        _, rep = glm.classify(Wg, "gmm")
    # the same optimum: the oracle's L_i at the GPU's fitted rows against its own optimum
    Wmix = Wg.copy()
    bmix = bg.copy()
    Wmix[rows] = fo["W"]
    bmix[rows] = fo["b"]
    Lo = oracle.eval_rows(w["offs"], w["bins"], T, w["dt"], w["tau"], Wmix, bmix, rows, grad=False)["L"]
    Lg = oracle.eval_rows(w["offs"], w["bins"], T, w["dt"], w["tau"], Wg, bg, rows, grad=False)["L"]
    gap = (Lo - Lg) / np.abs(Lo)
    dW = np.abs(Wg[rows] - fo["W"])
    print(f"{prec} subset fit: L_i gap oracle - GPU max {gap.max():.2e} (min {gap.min():.2e}, mean {gap.mean():.2e}), "
          f"max |dW| {dW.max():.2e}")
    assert np.all(gap <= gap_bound) and np.all(gap >= gap_low)
    # labels under the GPU fit's mixture model, except entries near a decision boundary
    pi, mu, var = np.array(rep["weights"]), np.array(rep["centers"]), np.array(rep["variances"])
    grid = np.linspace(mu[0], mu[2], 200001)
    lab_grid = gmm_assign(grid, pi, mu, var)
    bounds = grid[1:][np.diff(lab_grid) != 0]
    off = np.ones((len(rows), n), dtype=bool)
    off[np.arange(len(rows)), rows] = False
    lg = gmm_assign(Wg[rows][off], pi, mu, var)
    lo = gmm_assign(fo["W"][off], pi, mu, var)
    band = 10 * dW.max() + (grid[1] - grid[0])
    near = np.min(np.abs(Wg[rows][off][:, None] - bounds[None, :]), axis=1) < band
    differ = lg != lo
    print(f"{prec} labels: {int(differ.sum())} of {lg.size} differ, all within the ambiguous band: "
          f"{bool(np.all(near[differ]))} ({int(near.sum())} entries in the band)")
    assert np.all(near[differ])
