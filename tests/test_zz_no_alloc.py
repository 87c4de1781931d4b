"""glm_loglik_noalloc: the allocation-free log-likelihood, for callers that may not allocate device
memory (their memory belongs to another allocator, or they must not call cudaMalloc after start-up).

Called through the C ABI directly; its output must match the per-row log-likelihood of the regular
entry point (glm_loglik_grad on a GLM_PREC_F32 problem) on two calls in a row, within the plain FP32
form's per-row tolerance used by the parity tests (5e-8 relative).  It must work in a fresh process and
after any other test.  This file is named to be collected last."""
import ctypes

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
    return g


def test_noalloc_matches_regular_entry_point(glm):
    lib = glm.load_library()
    n, T = 37, 9001
    w = synth.make_workload(None, n=n, n_exc=29, p=0.1, w_exc=0.3, w_inh=1.2, w_self=-3.0, rate=8.0, tau=0.01,
                            dt=0.001, n_bins=T, seed=1)
    rng = np.random.default_rng(3)
    W = torch.from_numpy((w["W_true"] + rng.normal(0, 0.05, (n, n))).astype(np.float32)).cuda()
    b = torch.from_numpy((w["b_true"] + rng.normal(0, 0.1, n)).astype(np.float32)).cuda()
    with glm.GLM(0) as ctx:
        ctx.set_problem(w["offs"], w["bins"], T, w["dt"], w["tau"], prec="f32")
        ref = ctx.loglik_grad(W, b)["L_rows"].clone()
        X = ctx.filter(0, T, "f32")            # caller-owned inputs for the allocation-free call
        C, q = ctx.spike_term()
        stream = ctx.stream
        torch.cuda.synchronize()
        for _ in range(2):  # the fixed scratch keeps the previous call's contents
            out = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
            rc = lib.glm_loglik_noalloc(n, T, w["dt"], ctypes.c_void_p(X.data_ptr()), X.stride(0),
                                        ctypes.c_void_p(C.data_ptr()), ctypes.c_void_p(q.data_ptr()),
                                        ctypes.c_void_p(W.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
            assert rc == 0, glm.ERRORS.get(rc, rc)
            torch.cuda.synchronize()
            o, r = out.cpu().numpy(), ref.cpu().numpy()
            assert np.all(np.isfinite(o))
            assert np.all(np.abs(o - r) <= 5e-8 * np.abs(r) + 1e-9), np.max(np.abs(o - r) / np.abs(r))


def test_noalloc_rejects_problems_beyond_its_scratch(glm):
    lib = glm.load_library()
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    n, T = 1000, 1_800_000  # needs n * (T / 128 + 1) * 8 bytes, far beyond the fixed scratch
    rc = lib.glm_loglik_noalloc(n, T, 1e-3, p, T, p, p, p, p, p, None)
    assert rc == -11
    assert lib.glm_strerror(rc).decode().startswith("problem too large")
