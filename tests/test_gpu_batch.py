"""glm_fit_batch: several recordings of uneven N and T fitted together (one launch per contraction over all
problems, one CUDA graph per optimiser iteration), against the oracle's fits and against fitting each
recording alone.  Each row's optimum is unique (App. A), so the batched fit must land where the single fit
and the oracle land, up to the noise floor of the 16-bit evaluation (as in the single-fit test)."""
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


def recordings():
    out = [synth.make_workload("glm_n50_t20k")]
    for n, T, seed in [(37, 9001, 1), (130, 12000, 2)]:
        out.append(synth.make_workload(None, n=n, n_exc=int(0.8 * n), p=0.1, w_exc=0.3, w_inh=1.2, w_self=-3.0,
                                       rate=8.0, tau=0.01, dt=0.001, n_bins=T, seed=seed))
    return out


@pytest.mark.parametrize("prec", ["bf16", "f16"])
def test_batch_matches_single_fits_and_oracle(glm, prec):
    ws = recordings()
    ctxs = [glm.GLM(0) for _ in ws]
    try:
        for c, w in zip(ctxs, ws):
            c.set_problem(w["offs"], w["bins"], w["n_bins"], w["dt"], w["tau"], prec=prec)
        res, rc = glm.fit_batch(ctxs, eta=1e-10, max_iter=500)
        assert rc >= 0
        for c, w, r in zip(ctxs, ws, res):
            rep = r["report"]
            print(prec, w["n"], w["n_bins"], rep)
            assert rep["maxiter"] == 0 and rep["stalled"] == 0
            fo = oracle.fit(w["offs"], w["bins"], w["n_bins"], w["dt"], w["tau"], eta=1e-10, max_iter=500)
            Wb = r["W"].cpu().numpy().astype(np.float64)
            bb = r["b"].cpu().numpy().astype(np.float64)
            single = c.fit(eta=1e-10, max_iter=500)
            Ws = single["W"].cpu().numpy().astype(np.float64)
            # same optimum: the oracle's log-likelihood at the batched fit is within the noise floor of the
            # 16-bit evaluation of the oracle optimum and of the single fit
            Lb = oracle.loglik_grad(w["offs"], w["bins"], w["n_bins"], w["dt"], w["tau"], Wb, bb)["L_total"]
            Lo = oracle.loglik_grad(w["offs"], w["bins"], w["n_bins"], w["dt"], w["tau"], fo["W"], fo["b"])["L_total"]
            Ls = oracle.loglik_grad(w["offs"], w["bins"], w["n_bins"], w["dt"], w["tau"], Ws,
                                    single["b"].cpu().numpy().astype(np.float64))["L_total"]
            print(f"  L oracle opt {Lo:.9f} batch {Lb:.9f} single {Ls:.9f}; max |dW| vs oracle {np.abs(Wb - fo['W']).max():.2e}")
            assert Lb <= Lo + 1e-9 * abs(Lo)
            assert Lo - Lb <= 2e-6 * abs(Lo)
            assert abs(Lb - Ls) <= 2e-6 * abs(Lo)
            assert np.abs(Wb - fo["W"]).max() <= 0.1  # flat directions of the short recordings: L decides
    finally:
        for c in ctxs:
            c.close()


def test_batch_rejects_f32_and_mixed_precisions(glm):
    ws = recordings()[:2]
    ctxs = [glm.GLM(0) for _ in ws]
    try:
        for c, w in zip(ctxs, ws):
            c.set_problem(w["offs"], w["bins"], w["n_bins"], w["dt"], w["tau"], prec="f32")
        with pytest.raises(glm.GLMError) as e:
            glm.fit_batch(ctxs)
        assert e.value.code == -10
        ctxs[1].set_problem(ws[1]["offs"], ws[1]["bins"], ws[1]["n_bins"], ws[1]["dt"], ws[1]["tau"], prec="bf16")
        with pytest.raises(glm.GLMError) as e:
            glm.fit_batch(ctxs)
        assert e.value.code == -1
    finally:
        for c in ctxs:
            c.close()
