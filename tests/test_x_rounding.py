"""The case for one FP16 X (the default tensor-core form) on the host: the log-likelihood of the
balanced-network model with only the filtered trains X rounded to a 16-bit type, everything else in FP64
(the oracle's filter, products and sums), against the exact L.  FP16 keeps 11 significant bits of X and
moves L by a few 1e-7; BF16 keeps 8 and moves it by several 1e-6, past the 1e-6 bound of the 16-bit forms
(the kernel values a^k recur after every spike, so their rounding does not average out).  A network of 200
neurons over 60 000 bins with the weights perturbed from the generating ones."""
import numpy as np
import torch

import oracle
import synth


def test_fp16_x_meets_the_bound_bf16_does_not():
    w = synth.make_workload(None, n=200, n_exc=160, p=0.1, w_exc=0.2, w_inh=0.8, w_self=-6.25, rate=8.0,
                            tau=0.010, dt=0.001, n_bins=60000, seed=31)
    n, T, dt = w["n"], w["n_bins"], w["dt"]
    rng = np.random.default_rng(32)
    W = w["W_true"] + rng.normal(0, 0.02, (n, n))
    b = w["b_true"] + rng.normal(0, 0.05, n)
    X = oracle.filter(w["offs"], w["bins"], T, dt, w["tau"])
    spikes = [w["bins"][w["offs"][i]:w["offs"][i + 1]] for i in range(n)]

    def loglik(Xv):
        U = W @ Xv + b[:, None]
        return np.array([U[i, spikes[i]].sum() for i in range(n)]) - dt * np.exp(U).sum(axis=1)

    L = loglik(X)
    err = {}
    for name, dtype in (("f16", torch.float16), ("bf16", torch.bfloat16)):
        Xr = torch.from_numpy(X).to(dtype).double().numpy()
        err[name] = abs(loglik(Xr).sum() - L.sum()) / abs(L.sum())
    print(f"L relative change with X rounded: FP16 {err['f16']:.2e}, BF16 {err['bf16']:.2e}")
    assert err["f16"] <= 1e-6
    assert err["bf16"] >= 5 * err["f16"]
