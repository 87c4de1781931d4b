"""GPU parity of the continuous-time form (glm_set_problem_ct: event columns, exact interval integrals,
Eq. 8-14) against the FP64 continuous-time oracle, on off-grid spike times with the rates, weights and
sizes of the grid workloads (spikes of the grid generator moved uniformly inside their bins).

Tolerances are those of the grid's tensor-core forms: total log-likelihood relative 1e-6; per row
(|L_i| + q_i) x 3e-5 (BF16) or 4e-6 (FP16); gradient 2e-3 in the componentwise measure |dG_ij| /
(C_ij + (C_ij - G_ij)), the size of its two terms.  The column integrals themselves are FP32 Gauss-Legendre
sums accurate to ~3e-6 of F - D (tests/test_ct_interval.py)."""
import numpy as np
import pytest
import torch

import synth
from oracle import continuous as oc

pytestmark = pytest.mark.gpu

TOL = {"bf16": dict(total=1e-6, row=3e-5, grad=2e-3), "f16": dict(total=1e-6, row=4e-6, grad=2e-3)}


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


def workload(n, T, seed, delay):
    return synth.make_ct_workload(None, n=n, n_exc=max(1, int(0.8 * n)), p=0.1, w_exc=0.3, w_inh=1.2, w_self=-3.0,
                                  rate=8.0, tau=0.010, dt=0.001, n_bins=T, seed=seed, jitter_seed=seed + 11,
                                  delay=delay)


def params(w, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    n = w["n"]
    W = (scale * w["W_true"] + rng.normal(0, 0.05, (n, n)) * (scale != 0.0)).astype(np.float32)
    b = (w["b_true"] + rng.normal(0, 0.1, n)).astype(np.float32)
    return W, b


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def metric(G, G_ref, C_ref):
    mag = C_ref + (C_ref - G_ref)
    return float(np.max(np.abs(G - G_ref) / (mag + 1e-300)))


def check(ctx, w, W, b, prec, label, small=False):
    """small: a handful of spikes, where L is a near-cancellation of its spike and integral parts; the
    total is then measured against the size of those parts, sum_i (|L_i| + q_i)."""
    tol = TOL[prec]
    r = ctx.loglik_grad(to_dev(W), to_dev(b))
    ref = oc.loglik_grad(w["offs"], w["times"], w["t_begin"], w["t_end"], w["tau"], w["delay"],
                         W.astype(np.float64), b.astype(np.float64))
    q = ref["q"]
    scale = np.sum(np.abs(ref["L"]) + q) if small else abs(ref["L_total"])
    rel_tot = abs(r["L_total"] - ref["L_total"]) / scale
    Lr = r["L_rows"].cpu().numpy()
    rel_rows = float(np.max(np.abs(Lr - ref["L"]) / (np.abs(ref["L"]) + q + 1e-300)))
    g = metric(r["G"].cpu().numpy(), ref["G"], ref["C"])
    gb_err = float(np.max(np.abs(r["gb"].cpu().numpy() - ref["gb"]) / (q + np.abs(q - ref["gb"]) + 1e-300)))
    print(f"ct {label} {prec}: columns {ctx.columns()}, L total rel {rel_tot:.2e}, rows {rel_rows:.2e}, "
          f"grad {g:.2e}, gb {gb_err:.2e}")
    assert rel_tot <= tol["total"]
    assert rel_rows <= tol["row"]
    assert g <= tol["grad"]
    assert gb_err <= tol["row"]
    # spike term: S (V_hi + V_lo)^T, V to 16 significant bits (2^-17 relative), down to the smallest
    # FP16 subnormal (6e-8) for the decayed values of the FP16 form
    C, _ = ctx.spike_term()
    Cn = C.cpu().numpy()
    assert np.all(np.abs(Cn - ref["C"]) <= 3e-5 * ref["C"] + 1e-6)
    return r, ref


@pytest.mark.parametrize("prec", ["bf16", "f16"])
@pytest.mark.parametrize("n,T,seed,delay,scale", [(50, 20000, 0, 0.001, 1.0), (37, 9001, 1, 0.0015, 0.5),
                                                  (130, 5000, 2, 0.0, 1.0), (300, 20000, 4, 0.001, 1.0),
                                                  (9, 3000, 3, 0.002, 0.0)])
def test_ct_loglik_grad_matches_oracle(ctx, prec, n, T, seed, delay, scale):
    """Ragged N and column counts, several 128 x 256 tiles, zero delay (a spike and the arrivals at its
    own time share a column), and W = 0 (U = b: the u = 0 limit of every column)."""
    w = workload(n, T, seed, delay)
    W, b = params(w, seed + 100, scale)
    ctx.set_problem_ct(w["offs"], w["times"], w["t_begin"], w["t_end"], w["tau"], w["delay"], prec=prec)
    check(ctx, w, W, b, prec, f"n={n} T={T} d={delay}")


def test_ct_edge_cases(ctx):
    """Silent rows, coincident spike times across rows, a spike at t_begin, arrivals past t_end, one row."""
    rng = np.random.default_rng(5)
    t0, t1 = 2.0, 5.0
    rows = [np.sort(rng.uniform(t0, t1, 40)), np.zeros(0), np.sort(rng.uniform(t0, t1, 25)), np.zeros(0)]
    shared = np.array([2.5, 3.125, 4.75])
    rows[0] = np.unique(np.concatenate([rows[0], shared, [t0, t1 - 1e-4]]))
    rows[2] = np.unique(np.concatenate([rows[2], shared]))
    offs = np.zeros(5, dtype=np.int64)
    offs[1:] = np.cumsum([len(r) for r in rows])
    times = np.concatenate(rows)
    W = np.array([[-2.0, 0.0, 0.5, 0.0], [0.3, 0.0, -0.8, 0.0], [0.4, 0.0, -1.5, 0.0], [0.0, 0.0, 0.0, 0.0]],
                 dtype=np.float32)
    b = np.log(np.array([12.0, 3.0, 8.0, 1.0])).astype(np.float32)
    w = dict(offs=offs, times=times, t_begin=t0, t_end=t1, tau=0.02, delay=0.0015)
    for prec in ("bf16", "f16"):
        ctx.set_problem_ct(offs, times, t0, t1, 0.02, 0.0015, prec=prec)
        check(ctx, w, W, b, prec, "edge", small=True)
    # one neuron
    offs1 = np.array([0, 3], dtype=np.int64)
    times1 = np.array([0.01, 0.02, 0.5])
    w1 = dict(offs=offs1, times=times1, t_begin=0.0, t_end=1.0, tau=0.01, delay=0.001)
    ctx.set_problem_ct(offs1, times1, 0.0, 1.0, 0.01, 0.001, prec="bf16")
    check(ctx, w1, np.array([[-1.0]], np.float32), np.array([1.0], np.float32), "bf16", "single", small=True)


def test_ct_new_tau_and_determinism(ctx):
    w = workload(64, 8000, 6, 0.001)
    W, b = params(w, 9)
    ctx.set_problem_ct(w["offs"], w["times"], w["t_begin"], w["t_end"], w["tau"], w["delay"], prec="bf16")
    a = ctx.loglik_grad(to_dev(W), to_dev(b))
    a = {k: (v.clone() if torch.is_tensor(v) else v) for k, v in a.items()}
    c = ctx.loglik_grad(to_dev(W), to_dev(b))
    assert a["L_total"] == c["L_total"] and torch.equal(a["G"], c["G"])
    ctx.prepare(0.02)  # column decays, filter and spike term for the new tau
    w2 = dict(w, tau=0.02)
    check(ctx, w2, W, b, "bf16", "tau=0.02")


def test_ct_grid_aligned_times_match_the_grid_spike_term(ctx):
    """Times on the grid and a one-bin delay: the spike term of the event columns equals the grid's.  The
    bin width is a power of two, so that bin * dt + dt is exactly (bin + 1) * dt and an arrival coincides
    with a spike one bin later exactly, as on the grid."""
    dt = 2.0 ** -10
    g = synth.make_workload(None, n=40, n_exc=32, p=0.1, w_exc=0.3, w_inh=1.2, w_self=-3.0, rate=8.0, tau=0.01,
                            dt=dt, n_bins=6000, seed=8)
    times = g["bins"].astype(np.float64) * dt
    ctx.set_problem(g["offs"], g["bins"], 6000, dt, g["tau"], prec="bf16")
    Cg, _ = ctx.spike_term()
    Cg = Cg.cpu().numpy()
    ctx.set_problem_ct(g["offs"], times, 0.0, 6000 * dt, g["tau"], dt, prec="bf16")
    Cc, _ = ctx.spike_term()
    Cc = Cc.cpu().numpy()
    print(f"grid-aligned spike term: max rel difference {np.max(np.abs(Cc - Cg) / (Cg + 1e-12)):.2e}")
    # both are sums of V_hi + V_lo, each value to 2^-17 relative, rounded by two different scans
    assert np.all(np.abs(Cc - Cg) <= 3e-5 * Cg + 1e-8)


def test_ct_error_paths(glm, ctx):
    offs = np.array([0, 2], dtype=np.int64)
    with pytest.raises(glm.GLMError) as e:
        ctx.set_problem_ct(offs, np.array([0.2, 0.1]), 0.0, 1.0, 0.01, 0.001, prec="bf16")
    assert e.value.code == -2  # UNSORTED_SPIKES
    with pytest.raises(glm.GLMError) as e:
        ctx.set_problem_ct(offs, np.array([0.1, 1.0]), 0.0, 1.0, 0.01, 0.001, prec="bf16")
    assert e.value.code == -3  # SPIKE_OUT_OF_RANGE
    with pytest.raises(glm.GLMError) as e:
        ctx.set_problem_ct(offs, np.array([0.1, 0.2]), 0.0, 1.0, 0.01, 0.001, prec="f32")
    assert e.value.code == -10  # UNSUPPORTED
    with pytest.raises(glm.GLMError):
        ctx.set_problem_ct(offs, np.array([0.1, 0.2]), 0.0, 1.0, 0.01, -0.001, prec="bf16")
    ctx.set_problem_ct(offs, np.array([0.1, 0.2]), 0.0, 1.0, 0.01, 0.001, prec="bf16")
    W, b = to_dev(np.zeros((1, 1), np.float32)), to_dev(np.zeros(1, np.float32))
    assert ctx.loglik_grad(W, b, tau_grad=True)["gtau"] == 0.0  # W = 0: U = b does not depend on tau
    with pytest.raises(glm.GLMError) as e:
        ctx.filter(0, 2)
    assert e.value.code == -10  # UNSUPPORTED
    with pytest.raises(glm.GLMError) as e:
        glm.fit_batch([ctx])
    assert e.value.code == -10  # UNSUPPORTED: batched fits serve the grid form


def test_ct_fit_reaches_the_oracle_optimum(ctx):
    """glm_fit on event columns: at the returned (W, b) the oracle's continuous-time gradient is small
    against the size of its terms, and L is at least the oracle L at the generating weights."""
    w = workload(60, 60000, 12, 0.001)
    ctx.set_problem_ct(w["offs"], w["times"], w["t_begin"], w["t_end"], w["tau"], w["delay"], prec="bf16")
    res = ctx.fit(eta=1e-10, max_iter=300)
    W = res["W"].cpu().numpy().astype(np.float64)
    b = res["b"].cpu().numpy().astype(np.float64)
    ref = oc.loglik_grad(w["offs"], w["times"], w["t_begin"], w["t_end"], w["tau"], w["delay"], W, b)
    g = np.abs(ref["G"]) / (ref["C"] + (ref["C"] - ref["G"]) + 1e-300)
    q = ref["q"]
    print(f"ct fit: report {res['report']}, max rel gradient {g.max():.2e}, gb {np.max(np.abs(ref['gb']) / (q + 1)):.2e}")
    assert np.median(g) <= 1e-3 and g.max() <= 2e-2
    assert np.all(np.abs(ref["gb"]) <= 1e-2 * (q + 1))
    L0 = oc.loglik_grad(w["offs"], w["times"], w["t_begin"], w["t_end"], w["tau"], w["delay"], w["W_true"],
                        w["b_true"], grad=False)["L_total"]
    assert ref["L_total"] >= L0


def test_ct_cross_validation_recovers_tau(glm):
    """Cross-validation (Sec. 3.2 / 2.5) on off-grid times: fit on the first 60 % of the window, score on
    the rest, over tau; the data were generated with tau = 10 ms, which must win, and the best validation
    L must be the oracle's at the GPU fit."""
    w = workload(50, 40000, 31, 0.001)
    (tr, va) = glm.split_recording_ct(w["offs"], w["times"], w["t_begin"], w["t_end"], 24.0)
    taus = [0.005, 0.01, 0.02]
    with glm.GLM(0) as a, glm.GLM(0) as v:
        a.set_problem_ct(tr[0], tr[1], tr[2], tr[3], w["tau"], w["delay"], prec="bf16")
        v.set_problem_ct(va[0], va[1], va[2], va[3], w["tau"], w["delay"], prec="bf16")
        res = glm.cross_validate(a, v, [0.0], taus, eta=1e-10, max_iter=500)
        L = res["L_valid"]
        print("ct cross-validation", L.ravel())
        kt, ka = res["best"]
        assert taus[kt] == 0.01
        Lo = oc.loglik_grad(va[0], va[1], va[2], va[3], taus[kt], w["delay"],
                            res["W"].cpu().numpy().astype(np.float64), res["b"].cpu().numpy().astype(np.float64),
                            grad=False)["L_total"]
        assert abs(L[kt, ka] - Lo) <= 1e-6 * abs(Lo)


@pytest.mark.parametrize("prec", ["bf16", "f16"])
def test_ct_chunked_matches_stored(glm, prec):
    """Event columns recomputed chunk by chunk (glm_set_chunk_bins counts columns): every U-product tile sees
    the operands of the stored form, so L_i agree to the rounding of the final sums; E'V^T is summed over
    the chunks in another order (gradient to FP32 rounding of its partial sums); and the chunked form
    against the oracle at the usual bounds.  The chunk (8192 columns) cuts the ~40 000 columns into five
    chunks, the last one ragged."""
    w = workload(130, 20000, 5, 0.001)
    W, b = params(w, 6)
    args = (w["offs"], w["times"], w["t_begin"], w["t_end"], w["tau"], w["delay"])
    with glm.GLM(0) as a, glm.GLM(0) as c:
        a.set_problem_ct(*args, prec=prec)
        c.set_chunk_bins(8192)
        c.set_problem_ct(*args, prec=prec)
        M = c.columns()
        assert M == a.columns() and M > 4 * 8192
        ra = a.loglik_grad(to_dev(W), to_dev(b))
        La = ra["L_rows"].cpu().numpy()
        r, ref = check(c, w, W, b, prec, "chunked")
        Lc = r["L_rows"].cpu().numpy()
        q = ref["q"]
        assert np.all(np.abs(La - Lc) <= 1e-12 * (np.abs(La) + q))
        Ca = a.spike_term()[0].cpu().numpy()
        assert np.max(np.abs(ra["G"].cpu().numpy() - r["G"].cpu().numpy()) / (np.abs(Ca) + 1e-9)) <= 1e-5
        # a fit on the chunked columns reaches the stored form's optimum
        fa = a.fit(eta=1e-10, max_iter=300)
        fc = c.fit(eta=1e-10, max_iter=300)
        Wa = fa["W"].cpu().numpy().astype(np.float64)
        Wc = fc["W"].cpu().numpy().astype(np.float64)
        La_opt = oc.loglik_grad(*args, Wa, fa["b"].cpu().numpy().astype(np.float64), grad=False)["L_total"]
        Lc_opt = oc.loglik_grad(*args, Wc, fc["b"].cpu().numpy().astype(np.float64), grad=False)["L_total"]
        print(f"ct chunked {prec}: fits stored {La_opt:.9f} chunked {Lc_opt:.9f}")
        assert abs(La_opt - Lc_opt) <= 2e-6 * abs(La_opt)


def dtau_check(ctx, w, W, b, label):
    r = ctx.loglik_grad(to_dev(W), to_dev(b), tau_grad=True)
    ref = oc.loglik_grad(w["offs"], w["times"], w["t_begin"], w["t_end"], w["tau"], w["delay"],
                         W.astype(np.float64), b.astype(np.float64))
    scale = np.abs(ref["gtau_rows"]).sum()
    print(f"ct dL/dtau {label}: gpu {r['gtau']:.6e} oracle {ref['gtau']:.6e} scale {scale:.3e}")
    assert abs(r["gtau"] - ref["gtau"]) <= 1e-4 * scale
    return r, ref


@pytest.mark.parametrize("prec", ["bf16", "f16"])
@pytest.mark.parametrize("n,T,seed,delay", [(50, 20000, 0, 0.001), (37, 9001, 1, 0.0015), (130, 5000, 2, 0.0)])
def test_ct_dtau_matches_oracle(ctx, prec, n, T, seed, delay):
    """dL/dtau of the continuous-time form (the oracle's derivative is pinned to differences of the model's
    definition) within 1e-4 of the sum of the rows' contributions, as on the grid."""
    w = workload(n, T, seed, delay)
    W, b = params(w, seed + 1)
    ctx.set_problem_ct(w["offs"], w["times"], w["t_begin"], w["t_end"], w["tau"], w["delay"], prec=prec)
    r, _ = dtau_check(ctx, w, W, b, f"{prec} n={n} T={T} d={delay}")
    r2 = ctx.loglik_grad(to_dev(W), to_dev(b), tau_grad=True)
    assert r2["gtau"] == r["gtau"]  # deterministic


def test_ct_dtau_long_gaps_and_chunks(glm):
    """Silent stretches make columns of 5 tau (1 - a = 0.99: the closed form of dF/dtau) and of 200 tau
    (a = 0 in FP32: the decay chain restarts); the same recording with its columns in chunks gives the
    same dL/dtau."""
    w = workload(60, 6000, 7, 0.001)
    times, offs = w["times"].copy(), w["offs"]
    # a 50 ms gap after 2 s and a 2 s gap after 4 s: every later spike moves
    times = np.where(times >= 2.0, times + 0.05, times)
    times = np.where(times >= 4.05, times + 2.0, times)
    w = dict(w, times=times, t_end=w["t_end"] + 2.05)
    W, b = params(w, 8)
    args = (w["offs"], w["times"], w["t_begin"], w["t_end"], w["tau"], w["delay"])
    with glm.GLM(0) as a, glm.GLM(0) as c:
        a.set_problem_ct(*args, prec="f16")
        ra, _ = dtau_check(a, w, W, b, "gaps")
        c.set_chunk_bins(4096)
        c.set_problem_ct(*args, prec="f16")
        rc = c.loglik_grad(to_dev(W), to_dev(b), tau_grad=True)
        assert rc["gtau"] == pytest.approx(ra["gtau"], rel=1e-12, abs=1e-9)
