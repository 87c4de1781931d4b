"""glm_loglik_noalloc: the allocation-free log-likelihood, for callers that may not allocate device
memory (their memory belongs to another allocator, or they must not call cudaMalloc after start-up).

Called through the C ABI directly; its output must match the per-row log-likelihood of the regular
entry point (glm_loglik_grad on a GLM_PREC_F32 problem) on two calls in a row, within the plain FP32
form's per-row tolerance used by the parity tests (5e-8 relative), and the FP64 oracle within the same
bound.  Cases: one row tile with packed X; several row tiles (n not a multiple of 128) with X sliced
from a wider buffer (ldx > n_bins) and biases below the exp split at -60; a problem exactly at the
scratch limit.  Later calls must commit no device memory.  It must work in a fresh process and after
any other test.  This file is named to be collected last."""
import ctypes

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


def call_noalloc(lib, n, T, dt, X, C, q, W, b, out, stream):
    return lib.glm_loglik_noalloc(n, T, dt, ctypes.c_void_p(X.data_ptr()), X.stride(0),
                                  ctypes.c_void_p(C.data_ptr()), ctypes.c_void_p(q.data_ptr()),
                                  ctypes.c_void_p(W.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                  ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))


CASES = [
    # n, n_bins, extra columns of the X buffer (ldx = n_bins + extra), rows given a bias below -60
    (37, 9001, 0, 0),
    (150, 7000, 77, 5),
]


@pytest.mark.parametrize("n,T,extra,n_low", CASES)
def test_noalloc_matches_regular_entry_point(glm, n, T, extra, n_low):
    lib = glm.load_library()
    w = synth.make_workload(None, n=n, n_exc=int(0.8 * n), p=0.1, w_exc=0.3, w_inh=1.2, w_self=-3.0, rate=8.0,
                            tau=0.01, dt=0.001, n_bins=T, seed=1)
    rng = np.random.default_rng(3)
    Wn = (w["W_true"] + rng.normal(0, 0.05, (n, n))).astype(np.float32)
    bn = (w["b_true"] + rng.normal(0, 0.1, n)).astype(np.float32)
    bn[rng.choice(n, n_low, replace=False)] = rng.uniform(-75.0, -61.0, n_low).astype(np.float32)
    W = torch.from_numpy(Wn).cuda()
    b = torch.from_numpy(bn).cuda()
    with glm.GLM(0) as ctx:
        ctx.set_problem(w["offs"], w["bins"], T, w["dt"], w["tau"], prec="f32")
        ref = ctx.loglik_grad(W, b)["L_rows"].cpu().numpy()
        Xw = torch.full((n, T + extra), float("nan"), dtype=torch.float32, device="cuda")
        X = ctx.filter(0, T, "f32", out=Xw[:, :T])  # caller-owned inputs for the allocation-free call
        assert X.stride(0) == T + extra
        C, q = ctx.spike_term()
        stream = ctx.stream
        outs = [torch.full((n,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(3)]
        torch.cuda.synchronize()
        free = []
        for k in range(3):  # the fixed scratch keeps the previous call's contents
            free.append(torch.cuda.mem_get_info()[0])
            rc = call_noalloc(lib, n, T, w["dt"], X, C, q, W, b, outs[k], stream)
            assert rc == 0, glm.ERRORS.get(rc, rc)
            torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
    # the first call may commit the fixed array (lazy module loading); later calls commit nothing
    assert free[1] == free[2] == free[3], free
    orc = oracle.eval_rows(w["offs"], w["bins"], T, w["dt"], w["tau"], Wn.astype(np.float64),
                           bn.astype(np.float64), grad=False)
    qh = np.diff(w["offs"]).astype(np.float64)
    for out in outs[1:]:
        o = out.cpu().numpy()
        assert np.all(np.isfinite(o))
        assert np.all(np.abs(o - ref) <= 5e-8 * np.abs(ref) + 1e-9), np.max(np.abs(o - ref) / np.abs(ref))
        assert np.all(np.abs(o - orc["L"]) <= 5e-8 * (np.abs(orc["L"]) + qh)), \
            np.max(np.abs(o - orc["L"]) / (np.abs(orc["L"]) + qh))


def test_noalloc_at_the_scratch_limit(glm):
    """n (ceil(n_bins / 128) + 1) doubles exactly fill the 16 MiB array at n = 1000, n_bins = 268 288; one
    more tile of bins is refused and leaves the output untouched."""
    lib = glm.load_library()
    n, T = 1000, 268_288
    assert n * (-(-T // 128) + 1) * 8 <= 16 << 20 < n * (-(-(T + 128) // 128) + 1) * 8
    w = synth.make_workload("glm_n1000_t1800s", n_bins=T)
    rng = np.random.default_rng(5)
    W = torch.from_numpy((0.5 * w["W_true"] + rng.normal(0, 0.02, (n, n))).astype(np.float32)).cuda()
    b = torch.from_numpy(w["b_true"].astype(np.float32)).cuda()
    with glm.GLM(0) as ctx:
        ctx.set_problem(w["offs"], w["bins"], T, w["dt"], w["tau"], prec="f32")
        ref = ctx.loglik_grad(W, b, grad=False)["L_rows"].cpu().numpy()
        X = ctx.filter(0, T, "f32")
        C, q = ctx.spike_term()
        out = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        assert call_noalloc(lib, n, T, w["dt"], X, C, q, W, b, out, ctx.stream) == 0
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        assert np.all(np.abs(o - ref) <= 5e-8 * np.abs(ref) + 1e-9), np.max(np.abs(o - ref) / np.abs(ref))
        out2 = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        # refused before anything is read, so the X buffer need not hold the larger problem
        rc = lib.glm_loglik_noalloc(n, T + 128, w["dt"], ctypes.c_void_p(X.data_ptr()), T + 128,
                                    ctypes.c_void_p(C.data_ptr()), ctypes.c_void_p(q.data_ptr()),
                                    ctypes.c_void_p(W.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                    ctypes.c_void_p(out2.data_ptr()), ctypes.c_void_p(ctx.stream.cuda_stream))
        assert rc == -11
        torch.cuda.synchronize()
        assert torch.isnan(out2).all()


def test_noalloc_rejects_problems_beyond_its_scratch(glm):
    lib = glm.load_library()
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    n, T = 1000, 1_800_000  # needs n * (T / 128 + 1) * 8 bytes, far beyond the fixed scratch
    rc = lib.glm_loglik_noalloc(n, T, 1e-3, p, T, p, p, p, p, p, None)
    assert rc == -11
    assert lib.glm_strerror(rc).decode().startswith("problem too large")
