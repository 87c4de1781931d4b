"""FP64 oracle for Ward's minimum-variance hierarchical clustering of neurons by their synaptic weights
(Sec. 3.4.2: clustering the reconstructed connectivity by outgoing weights, the columns of W, or by
incoming weights, its rows; Ward 1963).

TEST INFRASTRUCTURE ONLY, under the same rule as the rest of ``oracle``: only the test suite,
``__graft_entry__.smoke()`` and the benchmark's CPU leg may import it.

Every neuron k is a point x_k (its column W[:, k] or its row W[k, :]).  Starting from singletons, each step
merges the two clusters A, B whose union raises the total within-cluster sum of squares the least,
  Delta(A, B) = |A| |B| / (|A| + |B|) ||mean_A - mean_B||^2,
computed here from the cluster means themselves (no update formula).  The merge height is
sqrt(2 Delta), the Euclidean form in which SciPy's linkage (the paper's tool) reports Ward merges.  The
result is a linkage matrix in SciPy's layout: row s = (id_a, id_b, height, size) with ids < n the points
and n + s' the cluster formed at step s', the smaller id first.  Pins: ``tests/test_ward_oracle_pins.py``.
"""
from __future__ import annotations

import numpy as np


def features(W, by: str = "out", subset=None) -> np.ndarray:
    """Points to cluster: columns of W (outgoing weights, by='out') or rows (incoming, by='in'), for the
    neurons in `subset` (all by default)."""
    W = np.asarray(W, dtype=np.float64)
    idx = np.arange(W.shape[0]) if subset is None else np.asarray(subset)
    return (W[:, idx].T if by == "out" else W[idx, :]).copy()


def ward_linkage(X) -> np.ndarray:
    """Greedy Ward merges of the rows of X (FP64), O(n^3) in the number of points."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    means = {k: X[k].copy() for k in range(n)}
    sizes = {k: 1 for k in range(n)}
    Z = np.zeros((n - 1, 4))
    for s in range(n - 1):
        ids = sorted(means)
        M = np.array([means[k] for k in ids])
        c = np.array([sizes[k] for k in ids], dtype=np.float64)
        sq = ((M[:, None, :] - M[None, :, :]) ** 2).sum(axis=2)
        delta = (c[:, None] * c[None, :] / (c[:, None] + c[None, :])) * sq
        np.fill_diagonal(delta, np.inf)
        a, b = np.unravel_index(np.argmin(delta), delta.shape)
        ia, ib = ids[a], ids[b]
        if ia > ib:
            ia, ib = ib, ia
        na, nb = sizes[ia], sizes[ib]
        Z[s] = (ia, ib, np.sqrt(2.0 * delta[a, b]), na + nb)
        means[n + s] = (na * means.pop(ia) + nb * means.pop(ib)) / (na + nb)
        sizes[n + s] = na + nb
        del sizes[ia], sizes[ib]
    return Z


def cut(Z, n: int, k: int) -> np.ndarray:
    """Cluster labels (0 .. k-1, numbered by each cluster's smallest member) after the first n - k merges."""
    parent = list(range(2 * n - 1))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for s in range(n - k):
        a, b = int(Z[s, 0]), int(Z[s, 1])
        parent[find(a)] = n + s
        parent[find(b)] = n + s
    roots = [find(i) for i in range(n)]
    order = {}
    for r in roots:
        order.setdefault(r, len(order))
    return np.array([order[r] for r in roots])
