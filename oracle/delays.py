"""FP64 oracle for per-neuron time constants and delays on the grid (Sec. 2.2: the kernel h_i belongs to
the target neuron, with its own tau_i; Sec. 2.4, Eq. 15: every source train is shifted by the delay with
which it reaches the target).

TEST INFRASTRUCTURE ONLY, under the same rule as the rest of ``oracle``: only the test suite,
``__graft_entry__.smoke()`` and the benchmark's CPU leg may import it.

Row i has (tau_i, d_i), d_i >= 1 bins.  A spike of neuron j in bin s reaches i in bin s + d_i:
  X^(i)_j[t] = sum over spikes s of j with s + d_i <= t of a_i^(t - d_i - s),   a_i = exp(-dt / tau_i)
  U_i[t]     = b_i + sum_j W_ij X^(i)_j[t]                                      (Eq. 3)
  L_i        = sum_{t in sp(i)} U_i[t] - dt sum_t exp(U_i[t])                   (Eq. 7 on the grid)
  dL/dW_ij   = sum_t R_i[t] X^(i)_j[t],  dL/db_i = sum_t R_i[t],  R = S - dt e^U (Eq. 12)
With d_i = 1 this is the grid model of ``oracle.loglik_grad``.  Rows of equal (tau, d) share X: it is the
grid filter (Eq. 13, ``oracle.filter``) of the trains shifted by d - 1 bins.

Self-delay (Sec. 2.4 and Sec. 3.1: the paper's own network has one transmission delay d for every
connection and a separate self-delay d_s for each neuron's action on itself): with ``self_delay_rows``
row i's own train reaches it after s_i bins while every other train arrives after d_i, so the diagonal
term of U_i uses X^(i,self)_i[t] = sum over spikes s of i with s + s_i <= t of a_i^(t - s_i - s), and
dL/dW_ii = sum_t R_i[t] X^(i,self)_i[t].  Pins: ``tests/test_delay_oracle_pins.py``.
"""
from __future__ import annotations

import numpy as np


def shift_trains(offs, bins, n_bins: int, shift: int):
    """The trains with every spike moved `shift` bins later; spikes pushed past the recording drop out."""
    offs = np.asarray(offs, dtype=np.int64)
    bins = np.asarray(bins, dtype=np.int64)
    n = len(offs) - 1
    rows, new_offs = [], np.zeros(n + 1, dtype=np.int64)
    for i in range(n):
        s = bins[offs[i]:offs[i + 1]] + shift
        s = s[s < n_bins]
        rows.append(s)
        new_offs[i + 1] = new_offs[i] + len(s)
    return new_offs, (np.concatenate(rows) if rows else np.zeros(0)).astype(np.int32)


def loglik_grad_classes(offs, bins, n_bins: int, dt: float, tau_rows, delay_rows, W, b,
                        self_delay_rows=None) -> dict:
    """L_i, L, dL/dW, dL/db with row i's own tau_i and delay d_i, and (when given) its self-delay s_i for
    the diagonal term (FP64)."""
    from . import filter as grid_filter
    offs = np.asarray(offs, dtype=np.int64)
    bins = np.asarray(bins, dtype=np.int64)
    W = np.asarray(W, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    tau_rows = np.asarray(tau_rows, dtype=np.float64)
    delay_rows = np.asarray(delay_rows, dtype=np.int64)
    n = len(offs) - 1
    self_rows = delay_rows if self_delay_rows is None else np.asarray(self_delay_rows, dtype=np.int64)
    L = np.zeros(n)
    G = np.zeros((n, n))
    gb = np.zeros(n)
    for tau, d in sorted(set(zip(tau_rows.tolist(), delay_rows.tolist()))):
        rows = np.nonzero((tau_rows == tau) & (delay_rows == d))[0]
        so, sb = shift_trains(offs, bins, n_bins, int(d) - 1)
        X = grid_filter(so, sb, n_bins, dt, tau)
        for i in rows:
            # row i's own train, as it reaches row i: shifted by its self-delay instead of d
            own_o = np.array([0, offs[i + 1] - offs[i]], dtype=np.int64)
            oo, ob = shift_trains(own_o, bins[offs[i]:offs[i + 1]], n_bins, int(self_rows[i]) - 1)
            Xi = X.copy() if self_rows[i] != d else X
            if self_rows[i] != d:
                Xi[i] = grid_filter(oo, ob, n_bins, dt, tau)[0]
            U = b[i] + W[i] @ Xi
            S = np.zeros(n_bins)
            S[bins[offs[i]:offs[i + 1]]] = 1.0
            E = dt * np.exp(U)
            L[i] = (S * U).sum() - E.sum()
            R = S - E
            G[i] = Xi @ R
            gb[i] = R.sum()
    return dict(L=L, L_total=float(L.sum()), G=G, gb=gb)
