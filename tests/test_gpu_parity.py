"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, element by element, on seeded
inputs that span several tiles and ragged tails, plus edge cases, error paths and a sampled check at the
full N = 1000, 1.8M-bin size.

Tolerances.  Plain FP32 form: filtered trains within a few FP32 ulps; spike term relative 5e-7 (a sum
of FP32 X values, each rounded once or twice); log-likelihood relative 1e-9 (total) and, per row, 5e-8 of
(|L_i| + q_i), the size of its terms (L_i itself can cross zero).  The total-L bound needs X without a
systematic rounding error: the kernel values e^{-k dt/tau} (Eq. 13) recur after every spike, so a scan
that rounds the chain 1, a, a^2, ... repeatedly biases X by ~0.6 ulp (about 2e-9 in L); the scan
takes each power rounded once.  It also needs the spike part of L in FP64 from the spike term C
(q_i b_i + sum_j W_ij C_ij): summing the FP32-accumulated U over the spike bins instead adds ~1e-9.
gradient componentwise relative 1e-5 against the size of its two terms, |dG_ij| / (C_ij + dt sum_t
e^{U_i} X_j).  Tensor-core forms (X and the rates in BF16 or FP16, W as hi + lo): total log-likelihood
relative 1e-6, gradient 2e-3 in the same componentwise measure.  Per row, the X rounding error
(relative 2^-9 for BF16, 2^-12 for FP16, random over bins; per-row errors are also measured against
(|L_i| + q_i)) bounds the integral term's error by about
sqrt(T) * dt e^U * 2^-9 |W X|: the per-row bounds below (3e-5 BF16, 4e-6 FP16) follow from that.
"""
import math

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
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return g


@pytest.fixture(scope="module")
def ctx(glm):
    c = glm.GLM(0)
    yield c
    c.close()


def workload(n, T, seed, *, rate=8.0, tau=0.010, dt=0.001, p=0.1, w_exc=0.3, w_inh=1.2, w_self=-3.0):
    return synth.make_workload(None, n=n, n_exc=max(1, int(0.8 * n)), p=p, w_exc=w_exc, w_inh=w_inh, w_self=w_self,
                               rate=rate, tau=tau, dt=dt, n_bins=T, seed=seed)


def oracle_spike_term(w, X):
    n = w["n"]
    C = np.zeros((n, n))
    for i in range(n):
        s = w["bins"][w["offs"][i]:w["offs"][i + 1]]
        C[i] = X[:, s].sum(axis=1)
    return C


def metric10(G, G_ref, C_ref):
    mag = C_ref + (C_ref - G_ref)  # C + dt sum_t e^U X, both terms >= 0
    return float(np.max(np.abs(G - G_ref) / (mag + 1e-300)))


def params(w, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    n = w["n"]
    W = (scale * w["W_true"] + rng.normal(0, 0.05, (n, n))).astype(np.float32)
    b = (w["b_true"] + rng.normal(0, 0.1, n)).astype(np.float32)
    return W, b


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# --------------------------------------------------------------------------- a0/a1 filter scan

@pytest.mark.parametrize("n,T,seed", [(37, 9001, 1), (8, 256, 2), (1, 1, 3), (13, 300, 4), (50, 20000, 0)])
def test_filter_matches_oracle(ctx, n, T, seed):
    w = workload(n, T, seed)
    ctx.set_problem(w["offs"], w["bins"], T, w["dt"], w["tau"], prec="f32")
    X = ctx.filter(0, T, "f32").cpu().numpy().astype(np.float64)
    Xo = oracle.filter(w["offs"], w["bins"], T, w["dt"], w["tau"])
    assert np.allclose(X, Xo, rtol=2e-6, atol=1e-7), np.max(np.abs(X - Xo))
    # 16-bit outputs are the FP32 values rounded once
    for dt_name, eps in (("bf16", 2.0 ** -8), ("f16", 2.0 ** -11)):
        Xh = ctx.filter(0, T, dt_name).float().cpu().numpy()
        assert np.all(np.abs(Xh - Xo) <= eps * np.abs(Xo) + 1e-6), dt_name


def test_filter_range_and_bursts(ctx):
    T, n = 12000, 6
    rows = [np.arange(1000, 1400, dtype=np.int32),            # 400 spikes in consecutive bins (bursts > 32/segment)
            np.array([], dtype=np.int32),                      # silent
            np.array([0, T - 1], dtype=np.int32),              # first and last bin
            np.arange(255, T, 256, dtype=np.int32),            # on segment boundaries
            np.arange(4095, T, 4096, dtype=np.int32),          # on chunk boundaries
            np.sort(np.random.default_rng(5).choice(T, 700, replace=False)).astype(np.int32)]
    offs = np.zeros(n + 1, dtype=np.int64)
    offs[1:] = np.cumsum([len(r) for r in rows])
    bins = np.concatenate(rows)
    dt, tau = 1e-3, 0.02
    ctx.set_problem(offs, bins, T, dt, tau, prec="f32")
    Xo = oracle.filter(offs, bins, T, dt, tau)
    X = ctx.filter(0, T, "f32").cpu().numpy()
    assert np.allclose(X, Xo, rtol=2e-6, atol=1e-6)
    out = torch.full((n, 5003), -7.0, dtype=torch.float32, device="cuda")
    ctx.filter(777, 5000, "f32", out=out)
    o = out.cpu().numpy()
    assert np.allclose(o[:, :5000], Xo[:, 777:5777], rtol=2e-6, atol=1e-6)
    assert np.all(o[:, 5000:] == -7.0)  # nothing written past t_len


# --------------------------------------------------------------------------- a2 spike term

@pytest.mark.parametrize("n,T,seed", [(37, 9001, 1), (50, 20000, 0), (70, 13000, 7)])
def test_spike_term_matches_oracle(ctx, n, T, seed):
    w = workload(n, T, seed)
    ctx.set_problem(w["offs"], w["bins"], T, w["dt"], w["tau"], prec="f32")
    C, q = ctx.spike_term()
    Xo = oracle.filter(w["offs"], w["bins"], T, w["dt"], w["tau"])
    Co = oracle_spike_term(w, Xo)
    assert np.array_equal(q.cpu().numpy(), np.diff(w["offs"]).astype(np.float64))
    assert np.allclose(C.cpu().numpy(), Co, rtol=5e-7, atol=1e-9)


# --------------------------------------------------------------------------- a3-a5, a7 log-likelihood and gradient

@pytest.mark.parametrize("n,T,seed,scale", [(50, 20000, 0, 1.0), (37, 9001, 1, 0.5), (130, 5000, 2, 1.0),
                                            (9, 700, 3, 0.0)])
def test_loglik_grad_f32_matches_oracle(ctx, n, T, seed, scale):
    w = workload(n, T, seed)
    W, b = params(w, seed + 100, scale)
    ctx.set_problem(w["offs"], w["bins"], T, w["dt"], w["tau"], prec="f32")
    r = ctx.loglik_grad(to_dev(W), to_dev(b))
    ref = oracle.loglik_grad(w["offs"], w["bins"], T, w["dt"], w["tau"], W.astype(np.float64), b.astype(np.float64))
    print(f"f32 n={n} T={T}: L total rel {abs(r['L_total'] - ref['L_total']) / abs(ref['L_total']):.2e}")
    assert abs(r["L_total"] - ref["L_total"]) <= 1e-9 * abs(ref["L_total"])
    Lr = r["L_rows"].cpu().numpy()
    assert np.all(np.abs(Lr - ref["L"]) <= 5e-8 * (np.abs(ref["L"]) + np.diff(w["offs"])))
    gb = r["gb"].cpu().numpy()
    q = np.diff(w["offs"]).astype(np.float64)
    assert np.all(np.abs(gb - ref["gb"]) <= 1e-8 * (q + np.abs(q - ref["gb"])) + 1e-9)
    C, _ = ctx.spike_term()
    assert metric10(r["G"].cpu().numpy(), ref["G"], C.cpu().numpy()) <= 1e-5


TC_TOL = {"bf16": dict(total=1e-6, row=3e-5, grad=2e-3), "f16": dict(total=1e-6, row=4e-6, grad=2e-3)}


@pytest.mark.parametrize("prec", ["bf16", "f16"])
@pytest.mark.parametrize("n,T,seed,scale", [(50, 20000, 0, 1.0), (37, 9001, 1, 0.5), (130, 5000, 2, 1.0),
                                            (300, 70000, 4, 1.0), (9, 700, 3, 0.0)])
def test_loglik_grad_tensor_core_matches_oracle(ctx, prec, n, T, seed, scale):
    """tcgen05 path: ragged N (tiles of 128 x 256 and 128 x 256 split-K), ragged T, more tiles than SMs."""
    tol = TC_TOL[prec]
    w = workload(n, T, seed)
    W, b = params(w, seed + 100, scale)
    ctx.set_problem(w["offs"], w["bins"], T, w["dt"], w["tau"], prec=prec)
    r = ctx.loglik_grad(to_dev(W), to_dev(b))
    ref = oracle.loglik_grad(w["offs"], w["bins"], T, w["dt"], w["tau"], W.astype(np.float64), b.astype(np.float64))
    rel_tot = abs(r["L_total"] - ref["L_total"]) / abs(ref["L_total"])
    Lr = r["L_rows"].cpu().numpy()
    rel_rows = np.max(np.abs(Lr - ref["L"]) / (np.abs(ref["L"]) + np.diff(w["offs"])))
    C, _ = ctx.spike_term()
    g = metric10(r["G"].cpu().numpy(), ref["G"], C.cpu().numpy())
    print(f"{prec} n={n} T={T}: L total rel {rel_tot:.2e}, rows max rel {rel_rows:.2e}, grad {g:.2e}")
    assert rel_tot <= tol["total"]
    assert rel_rows <= tol["row"]
    assert g <= tol["grad"]
    q = np.diff(w["offs"]).astype(np.float64)
    assert np.all(np.abs(r["gb"].cpu().numpy() - ref["gb"]) <= tol["row"] * (q + np.abs(q - ref["gb"])) + 1e-9)


def test_tensor_core_deterministic(ctx):
    w = workload(130, 5000, 2)
    W, b = params(w, 7)
    ctx.set_problem(w["offs"], w["bins"], 5000, w["dt"], w["tau"], prec="bf16")
    a = ctx.loglik_grad(to_dev(W), to_dev(b))
    a = {k: (v.clone() if torch.is_tensor(v) else v) for k, v in a.items()}
    c = ctx.loglik_grad(to_dev(W), to_dev(b))
    assert a["L_total"] == c["L_total"]
    assert torch.equal(a["G"], c["G"])


def test_zero_spike_rows_and_single_neuron(ctx):
    T = 3000
    offs = np.array([0, 0, 40, 40], dtype=np.int64)   # rows 0 and 2 never spike
    bins = np.sort(np.random.default_rng(1).choice(T, 40, replace=False)).astype(np.int32)
    W = np.array([[0.0, 0.3, 0.0], [0.2, -1.0, 0.1], [0.0, 0.4, 0.0]], dtype=np.float32)
    b = np.array([0.5, 2.0, -1.0], dtype=np.float32)
    ctx.set_problem(offs, bins, T, 1e-3, 0.01, prec="f32")
    r = ctx.loglik_grad(to_dev(W), to_dev(b))
    ref = oracle.loglik_grad(offs, bins, T, 1e-3, 0.01, W.astype(np.float64), b.astype(np.float64))
    assert np.all(np.abs(r["L_rows"].cpu().numpy() - ref["L"]) <= 5e-8 * (np.abs(ref["L"]) + np.diff(offs)))
    assert np.allclose(r["G"].cpu().numpy(), ref["G"], rtol=1e-6, atol=1e-9)
    # one neuron, one bin
    ctx.set_problem(np.array([0, 1], dtype=np.int64), np.array([0], dtype=np.int32), 1, 1e-3, 0.01, prec="f32")
    r = ctx.loglik_grad(to_dev(np.array([[0.7]], np.float32)), to_dev(np.array([1.5], np.float32)))
    assert r["L_total"] == pytest.approx(1.5 - 1e-3 * math.exp(1.5), rel=1e-12)
    assert r["G"].item() == 0.0


def test_deterministic(ctx):
    w = workload(37, 9001, 1)
    W, b = params(w, 5)
    ctx.set_problem(w["offs"], w["bins"], 9001, w["dt"], w["tau"], prec="f32")
    a = ctx.loglik_grad(to_dev(W), to_dev(b))
    a = {k: (v.clone() if torch.is_tensor(v) else v) for k, v in a.items()}
    c = ctx.loglik_grad(to_dev(W), to_dev(b))
    assert a["L_total"] == c["L_total"]
    assert torch.equal(a["G"], c["G"]) and torch.equal(a["L_rows"], c["L_rows"])


def test_error_paths(glm, ctx):
    with pytest.raises(glm.GLMError) as e:
        ctx.set_problem(np.array([0, 2], np.int64), np.array([5, 5], np.int32), 10, 1e-3, 0.01)
    assert e.value.code == -2
    with pytest.raises(glm.GLMError) as e:
        ctx.set_problem(np.array([0, 1], np.int64), np.array([10], np.int32), 10, 1e-3, 0.01)
    assert e.value.code == -3
    with pytest.raises(glm.GLMError) as e:
        ctx.set_problem(np.array([0, 1], np.int64), np.array([3], np.int32), 10, -1e-3, 0.01)
    assert e.value.code == -1
    fresh = glm.GLM(0)
    with pytest.raises(glm.GLMError) as e:
        fresh.loglik_grad(torch.zeros((1, 1), device="cuda"), torch.zeros(1, device="cuda"))
    assert e.value.code == -9
    fresh.close()
    # exp(U) overflow is reported, not silently returned
    ctx.set_problem(np.array([0, 3], np.int64), np.array([1, 2, 3], np.int32), 10, 1e-3, 0.01)
    with pytest.raises(glm.GLMError) as e:
        ctx.loglik_grad(to_dev(np.array([[1e4]], np.float32)), to_dev(np.array([0.0], np.float32)))
    assert e.value.code == -6
    with pytest.raises(glm.GLMError) as e:
        ctx.loglik_grad(to_dev(np.array([[0.0]], np.float32)), to_dev(np.array([float("nan")], np.float32)))
    assert e.value.code == -6


def test_workspace_cap(glm):
    w = workload(37, 9001, 1)
    c = glm.GLM(0, workspace_cap=1 << 20)
    with pytest.raises(glm.GLMError) as e:
        c.set_problem(w["offs"], w["bins"], 9001, w["dt"], w["tau"])
    assert e.value.code == -4
    c.close()


# --------------------------------------------------------------------------- full size, sampled

@pytest.fixture(scope="module")
def full_size():
    return synth.make_workload("glm_n1000_t1800s")


def test_full_size_sampled_rows_bf16(ctx, full_size):
    """N = 1000, 1.8M bins, BF16 tensor-core path as the benchmark runs it; 4 rows checked by the oracle."""
    w = full_size
    T = w["n_bins"]
    W = w["W_true"].astype(np.float32)
    b = w["b_true"].astype(np.float32)
    ctx.set_problem(w["offs"], w["bins"], T, w["dt"], w["tau"], prec="bf16")
    r = ctx.loglik_grad(to_dev(W), to_dev(b))
    rows = np.array([0, 333, 801, 999], dtype=np.int32)
    ref = oracle.eval_rows(w["offs"], w["bins"], T, w["dt"], w["tau"], W.astype(np.float64), b.astype(np.float64),
                           rows)
    Lr = r["L_rows"].cpu().numpy()[rows]
    rel = np.abs(Lr - ref["L"]) / (np.abs(ref["L"]) + np.diff(w["offs"])[rows])
    C, _ = ctx.spike_term()
    g = metric10(r["G"].cpu().numpy()[rows], ref["G"], C.cpu().numpy()[rows])
    print(f"full-size bf16: rows rel {rel}, grad {g:.2e}")
    assert np.all(rel <= TC_TOL["bf16"]["row"])
    assert g <= TC_TOL["bf16"]["grad"]


def test_full_size_sampled_rows_f32(ctx, full_size):
    """N = 1000, 1.8M bins in the benchmark's launch configuration; the oracle checks 4 sampled rows."""
    w = full_size
    n, T = w["n"], w["n_bins"]
    W = w["W_true"].astype(np.float32)
    b = w["b_true"].astype(np.float32)
    ctx.set_problem(w["offs"], w["bins"], T, w["dt"], w["tau"], prec="f32")
    r = ctx.loglik_grad(to_dev(W), to_dev(b))
    rows = np.array([0, 333, 801, 999], dtype=np.int32)
    ref = oracle.eval_rows(w["offs"], w["bins"], T, w["dt"], w["tau"], W.astype(np.float64), b.astype(np.float64),
                           rows)
    Lr = r["L_rows"].cpu().numpy()[rows]
    assert np.all(np.abs(Lr - ref["L"]) <= 5e-8 * (np.abs(ref["L"]) + np.diff(w["offs"])[rows])), (Lr, ref["L"])
    C, _ = ctx.spike_term()
    Cr = C.cpu().numpy()[rows]
    assert metric10(r["G"].cpu().numpy()[rows], ref["G"], Cr) <= 1e-5
    assert np.all(np.abs(r["gb"].cpu().numpy()[rows] - ref["gb"]) <= 1e-7 * np.diff(w["offs"])[rows])


def test_same_shape_problem_reuses_buffers(glm, ctx):
    """A second recording of the same shape (neurons, bins, total spikes) renews only the spikes and the
    caches of the context; its results are those of a fresh context, bit for bit."""
    w = workload(60, 7000, 6)
    n, T = w["n"], 7000
    rows = [w["bins"][w["offs"][i]:w["offs"][i + 1]] for i in range(n)][::-1]  # same total, other rows
    offs2 = np.zeros(n + 1, dtype=np.int64)
    offs2[1:] = np.cumsum([len(r) for r in rows])
    bins2 = np.concatenate(rows).astype(np.int32)
    W, b = params(w, 9)
    for prec in ("bf16", "f32"):
        ctx.set_problem(w["offs"], w["bins"], T, w["dt"], w["tau"], prec=prec)
        ctx.loglik_grad(to_dev(W), to_dev(b))
        ctx.set_problem(offs2, bins2, T, w["dt"], 0.015, prec=prec)
        a = ctx.loglik_grad(to_dev(W), to_dev(b))
        with glm.GLM(0) as fresh:
            fresh.set_problem(offs2, bins2, T, w["dt"], 0.015, prec=prec)
            f = fresh.loglik_grad(to_dev(W), to_dev(b))
            assert a["L_total"] == f["L_total"]
            assert torch.equal(a["G"], f["G"]) and torch.equal(a["gb"], f["gb"])


def test_same_shape_recording_checked_on_device(glm, ctx):
    """A recording of the current problem's shape is checked on the device: a bin out of range or rows not
    strictly increasing give the errors (and messages) of the host check, and the problem stays as it was."""
    w = workload(40, 5000, 8)
    n, T = w["n"], 5000
    W, b = params(w, 4)
    ctx.set_problem(w["offs"], w["bins"], T, w["dt"], w["tau"], prec="bf16")
    before = ctx.loglik_grad(to_dev(W), to_dev(b))
    offs = w["offs"]
    r = int(np.argmax(np.diff(offs)))  # a row with several spikes
    k0 = int(offs[r])
    cases = []
    bad = w["bins"].copy(); bad[k0 + 1] = T                      # out of range
    cases.append((bad, glm.GLMError, "outside"))
    bad = w["bins"].copy(); bad[k0 + 1] = bad[k0]                # two spikes in one bin
    cases.append((bad, glm.GLMError, "strictly increasing"))
    bad = w["bins"].copy(); bad[k0 + 2] = -1                     # negative
    cases.append((bad, glm.GLMError, "outside"))
    for bins, exc, text in cases:
        with pytest.raises(exc) as e_dev:
            ctx.set_problem(offs, bins, T, w["dt"], w["tau"], prec="bf16")
        with glm.GLM(0) as fresh, pytest.raises(exc) as e_host:
            fresh.set_problem(offs, bins, T, w["dt"], w["tau"], prec="bf16")
        assert text in str(e_dev.value) and str(e_dev.value) == str(e_host.value)
        after = ctx.loglik_grad(to_dev(W), to_dev(b))
        assert after["L_total"] == before["L_total"] and torch.equal(after["G"], before["G"])
    # a row that starts lower than the previous row ends is valid (rows are checked separately)
    rows = [w["bins"][offs[i]:offs[i + 1]] for i in range(n)]
    assert any(len(rows[i]) and len(rows[i - 1]) and rows[i][0] <= rows[i - 1][-1] for i in range(1, n))
    ctx.set_problem(offs, w["bins"], T, w["dt"], w["tau"], prec="bf16")
    again = ctx.loglik_grad(to_dev(W), to_dev(b))
    assert again["L_total"] == before["L_total"]
