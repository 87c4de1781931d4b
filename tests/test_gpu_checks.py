"""Checks of the library itself, standing in for race detection and failure detection by a sanitizer: no
kernel reads a value it did not write, and a bounded device-side wait gives up, reports it and leaves the
context usable.

* Poisoned caches: every recomputed buffer filled with NaN bytes, then glm_prepare and an evaluation give
  the results of a fresh context bit for bit (grid BF16 and FP32, the chunked form, continuous time, a
  delayed row class).
* A wait on an mbarrier that nobody arrives on returns GLM_ERR_TIMEOUT after its limit, and the next
  evaluation on the same context is correct."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def glm():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1502_04993_gb300 as g
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return g


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def setups():
    w = synth.make_workload(None, n=70, n_exc=56, p=0.1, w_exc=0.3, w_inh=1.2, w_self=-3.0, rate=8.0, tau=0.01,
                            dt=0.001, n_bins=9000, seed=41)
    wc = synth.make_ct_workload(None, n=70, n_exc=56, p=0.1, w_exc=0.3, w_inh=1.2, w_self=-3.0, rate=8.0,
                                tau=0.01, dt=0.001, n_bins=9000, seed=42, delay=0.0013)
    grid = lambda c, prec: c.set_problem(w["offs"], w["bins"], 9000, 0.001, 0.01, prec=prec)
    return w, [
        ("bf16", lambda c: grid(c, "bf16")),
        ("f32", lambda c: grid(c, "f32")),
        ("chunked", lambda c: (c.set_chunk_bins(4096), grid(c, "bf16"))),
        ("delay3 rows 10-50", lambda c: (c.set_source_delay(3), grid(c, "bf16"), c.set_row_range(10, 50))),
        ("continuous", lambda c: c.set_problem_ct(wc["offs"], wc["times"], 0.0, wc["t_end"], 0.01, 0.0013,
                                                  prec="bf16")),
    ]


@pytest.mark.parametrize("k", range(5))
def test_poisoned_caches_give_the_fresh_result(glm, k):
    w, cases = setups()
    name, setup = cases[k]
    rng = np.random.default_rng(k)
    W = to_dev((w["W_true"] + rng.normal(0, 0.05, w["W_true"].shape)).astype(np.float32))
    b = to_dev(w["b_true"].astype(np.float32))
    with glm.GLM(0) as fresh, glm.GLM(0) as pois:
        setup(fresh)
        setup(pois)
        ref = fresh.loglik_grad(W, b)
        pois.poison_caches()
        pois.prepare()
        got = pois.loglik_grad(W, b)
        print(name, ref["L_total"], got["L_total"])
        assert np.isfinite(got["L_total"]) and got["L_total"] == ref["L_total"]
        assert torch.equal(got["G"], ref["G"]) and torch.equal(got["gb"], ref["gb"])
        assert torch.equal(got["L_rows"], ref["L_rows"])


def test_bounded_wait_gives_up_and_the_context_stays_usable(glm):
    w = synth.make_workload(None, n=30, n_exc=24, p=0.1, w_exc=0.3, w_inh=1.2, w_self=-3.0, rate=8.0, tau=0.01,
                            dt=0.001, n_bins=5000, seed=43)
    W = to_dev(w["W_true"].astype(np.float32))
    b = to_dev(w["b_true"].astype(np.float32))
    with glm.GLM(0) as c:
        c.set_problem(w["offs"], w["bins"], 5000, 0.001, 0.01, prec="bf16")
        before = c.loglik_grad(W, b)["L_total"]
        assert c.check_wait_limit(0.05) == -7  # GLM_ERR_TIMEOUT
        assert c.loglik_grad(W, b)["L_total"] == before
