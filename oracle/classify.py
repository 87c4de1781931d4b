"""Oracle classification of reconstructed weights into excitatory / absent / inhibitory.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Follows the paper's two classifiers of the off-diagonal weights J_ij, i != j
(self-connections and biases are treated separately, Sec. 3.1):
  * k-means with k = 3 on the 1-D weight values (Sec. 3.3 / App. C.2), and
  * a 3-component Gaussian mixture fitted by expectation-maximisation
    (Sec. 3.1), initialised from the k-means solution.
Clusters are named by ascending mean: inhibitory (-1), absent (0),
excitatory (+1).  Errors are broken down as in Table 2 (FP, FN and ND = a
misclassification that contradicts Dale's law for the presynaptic neuron's
type), and the chance level of a random classifier is Eq. 20 (App. C.1).

Readings where the paper is silent: k-means starts at the 1st, 50th and 99th
percentiles (linear interpolation) and runs Lloyd steps until no assignment
changes; a point equidistant from two centroids joins the one nearer zero; the
GMM stops at a relative change of the mixture log-likelihood below 1e-12 or
after 1000 EM steps, with a variance floor of 1e-12; a posterior tie goes to
the component nearer zero.
"""
from __future__ import annotations

import math

import numpy as np

LABEL_INH, LABEL_ABSENT, LABEL_EXC = -1, 0, 1


def offdiag(W: np.ndarray) -> np.ndarray:
    n = W.shape[0]
    return W[~np.eye(n, dtype=bool)]


def _nearest(x: np.ndarray, c: np.ndarray) -> np.ndarray:
    d = np.abs(x[:, None] - c[None, :])
    best = d.min(axis=1, keepdims=True)
    tie_ok = d == best
    # among equally near centroids prefer the one with the smallest |c|
    pref = np.where(tie_ok, np.abs(c)[None, :], np.inf)
    return pref.argmin(axis=1)


def kmeans1d(x: np.ndarray, max_iter: int = 1000):
    """Lloyd's k-means with k = 3 on 1-D data; returns (centroids ascending, assignment)."""
    x = np.asarray(x, dtype=np.float64).ravel()
    c = np.percentile(x, [1.0, 50.0, 99.0])
    assign = _nearest(x, c)
    for _ in range(max_iter):
        for k in range(3):
            sel = assign == k
            if sel.any():
                c[k] = x[sel].mean()
        new = _nearest(x, c)
        if np.array_equal(new, assign):
            break
        assign = new
    order = np.argsort(c, kind="stable")
    rank = np.empty(3, dtype=np.int64)
    rank[order] = np.arange(3)
    return c[order], rank[assign]


def gmm1d(x: np.ndarray, max_iter: int = 1000, tol: float = 1e-12, var_floor: float = 1e-12, trace=None):
    """3-component 1-D Gaussian mixture by EM, initialised from k-means.

    Returns (weights, means, variances) sorted by mean, the posterior-argmax assignment and the final
    mixture log-likelihood.  ``trace``, when a list, receives the mixture log-likelihood of every EM
    iterate (each before its M step)."""
    x = np.asarray(x, dtype=np.float64).ravel()
    c, a = kmeans1d(x)
    pi = np.array([(a == k).mean() for k in range(3)])
    mu = c.copy()
    var = np.array([x[a == k].var() if (a == k).any() else 0.0 for k in range(3)])
    var = np.maximum(var, var_floor)
    pi = np.maximum(pi, 1e-300)
    prev = -np.inf
    ll = -np.inf
    for _ in range(max_iter):
        # E step (log domain)
        logp = (np.log(pi)[None, :] - 0.5 * np.log(2 * math.pi * var)[None, :]
                - 0.5 * (x[:, None] - mu[None, :]) ** 2 / var[None, :])
        mx = logp.max(axis=1, keepdims=True)
        lse = mx[:, 0] + np.log(np.exp(logp - mx).sum(axis=1))
        ll = lse.sum()
        if trace is not None:
            trace.append(float(ll))
        resp = np.exp(logp - lse[:, None])
        # M step
        nk = resp.sum(axis=0)
        pi = np.maximum(nk / x.size, 1e-300)
        mu = (resp * x[:, None]).sum(axis=0) / np.maximum(nk, 1e-300)
        var = np.maximum((resp * (x[:, None] - mu[None, :]) ** 2).sum(axis=0) / np.maximum(nk, 1e-300), var_floor)
        if np.isfinite(prev) and abs(ll - prev) <= tol * abs(ll):
            break
        prev = ll
    order = np.argsort(mu, kind="stable")
    pi, mu, var = pi[order], mu[order], var[order]
    return (pi, mu, var), gmm_assign(x, pi, mu, var), ll


def gmm_assign(x: np.ndarray, pi: np.ndarray, mu: np.ndarray, var: np.ndarray) -> np.ndarray:
    """Component of largest posterior for each point; a tie goes to the component whose mean is nearer 0."""
    x = np.asarray(x, dtype=np.float64).ravel()
    logp = (np.log(pi)[None, :] - 0.5 * np.log(2 * math.pi * var)[None, :]
            - 0.5 * (x[:, None] - mu[None, :]) ** 2 / var[None, :])
    best = logp.max(axis=1, keepdims=True)
    tie = logp == best
    pref = np.where(tie, np.abs(mu)[None, :], np.inf)
    return pref.argmin(axis=1)


def classify(W: np.ndarray, method: str = "gmm"):
    """Labels (n x n int8: -1 inhibitory, 0 absent, +1 excitatory; diagonal 0) and the cluster model."""
    W = np.asarray(W, dtype=np.float64)
    n = W.shape[0]
    x = offdiag(W)
    if method == "kmeans":
        c, assign = kmeans1d(x)
        model = dict(centroids=c)
    elif method == "gmm":
        (pi, mu, var), assign, ll = gmm1d(x)
        model = dict(weights=pi, means=mu, variances=var, loglik=ll)
    else:
        raise ValueError(method)
    lab = np.zeros((n, n), dtype=np.int8)
    lab[~np.eye(n, dtype=bool)] = (assign - 1).astype(np.int8)
    return lab, model


def truth_labels(W_true: np.ndarray) -> np.ndarray:
    n = W_true.shape[0]
    lab = np.sign(W_true).astype(np.int8)
    lab[np.eye(n, dtype=bool)] = 0
    return lab


def mer_breakdown(labels: np.ndarray, truth: np.ndarray, types: np.ndarray | None = None) -> dict:
    """Misclassification rate over the n(n-1) off-diagonal pairs (Eq. 20's denominator) and over n^2
    (Table 2's), with per-class errors, FP, FN and Dale's-law violations (ND)."""
    n = labels.shape[0]
    off = ~np.eye(n, dtype=bool)
    lab = labels[off].astype(np.int64)
    tru = truth[off].astype(np.int64)
    wrong = lab != tru
    out = dict(errors=int(wrong.sum()), mer=float(wrong.mean()), mer_n2=float(wrong.sum() / (n * n)))
    pre_type = None
    if types is not None:
        pre_type = np.broadcast_to(np.asarray(types, dtype=np.int64)[None, :], (n, n))[off]
    for name, c in (("exc", LABEL_EXC), ("inh", LABEL_INH), ("absent", LABEL_ABSENT)):
        fp = int(((lab == c) & (tru != c)).sum())
        fn = int(((tru == c) & (lab != c)).sum())
        d = dict(errors=fp + fn, fp=fp, fn=fn)
        if pre_type is not None and c != LABEL_ABSENT:
            # a connection labelled with the sign opposite to its presynaptic neuron's type
            nd = int((((lab == c) & (tru != c)) & (pre_type == -c)).sum())
            d["nd"] = nd
        out[name] = d
    return out


def chance_mer(p: float, f_exc: float) -> float:
    """Misclassification rate of a random classifier that keeps p, f_e and f_i = 1 - f_e (Eq. 20)."""
    f_inh = 1.0 - f_exc
    return p * (2.0 - p * (1.0 + f_exc ** 2 + f_inh ** 2))
