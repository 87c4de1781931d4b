"""FP64 oracle for the continuous-time log-likelihood (Sec. 2.3, Eq. 7-14), spike times off any grid.

TEST INFRASTRUCTURE ONLY, under the same rule as the rest of ``oracle``: only the test suite,
``__graft_entry__.smoke()`` and the benchmark's CPU leg may import it.

Model.  Spike k of neuron j is at t_jk in [t_begin, t_end); it reaches every neuron after one uniform
delay d >= 0 (Sec. 2.4, Eq. 15 with D_ij = d), so the network's arrival events are e = t_jk + d < t_end.
  v_j(t) = sum over arrivals e_jk <= t of exp(-(t - e_jk) / tau)          (Eq. 11 with h of Sec. 2.2, H(0) = 1)
  U_i(t) = b_i + sum_j W_ij v_j(t)                                          (Eq. 3; b_i is J_i0)
  L_i    = sum_k U_i(t_ik) - int_{t_begin}^{t_end} exp(U_i(t)) dt           (Eq. 2 / 7, exp link Eq. 5)

The steps follow the paper:
  * U_i - b_i and v_j just after every distinct arrival time by the key recurrence (Eq. 8) and its
    analogue for v (Eq. 13): decay by exp(-(gap) / tau), then add W_ij (resp. 1) per arriving spike of j;
  * U at a spike time: the value after the last arrival at or before it, decayed over the remaining gap;
  * the integral between consecutive events by the exponential-integral closed form (Eq. 10):
      int_0^D exp(b + u exp(-s / tau)) ds = e^b tau (Ei(u) - Ei(u a)),  a = exp(-D / tau),
    and its limit e^b D where u = 0 (no input yet, so U = b on the whole interval);
  * dL/dW_ij = sum_k v_j(t_ik) - e^{b_i} sum_m v_j(e_m) tau (e^u - e^{u a_m}) / u      (Eq. 12, 14)
    with the limit tau (1 - a_m) at u = 0, and dL/db_i = q_i - int exp(U_i)         (Eq. 12, j = 0).
  * dL/dtau (the paper chooses tau by cross-validation, Sec. 3.2, and gives no derivative; this is the
    exact derivative of the L above).  With y_j(t) = sum over arrivals (t - e) exp(-(t - e) / tau),
    dv_j/dtau = y_j / tau^2, and z = W y follows the recurrence of u: between events z decays with u and
    gains gap * u (z(e + g) = exp(-g / tau) (z(e) + g u(e))); arrivals add nothing to z.  Then
      dU_i(t)/dtau = z_i(t) / tau^2,
      d/dtau of one interval's integral e^b F(u, D) = e^b [G(u, D) z / tau^2 + (F - D e^{u a}) / tau]
    (G the interval weight above, dF/du = G; the explicit term by parts from F = int_0^D exp(u e^{-s/tau})
    ds), so dL_i/dtau = sum_k z_i(t_ik) / tau^2 - e^{b_i} sum_m [...].
Ei is scipy.special.expi (a library routine, FP64).  Pins: ``tests/test_ct_oracle_pins.py`` (adaptive
quadrature of the intensity built from its definition, finite differences, the grid form at grid-aligned
times, closed forms).
"""
from __future__ import annotations

import numpy as np
from scipy.special import expi


def arrival_events(offs, times, t_begin: float, t_end: float, delay: float):
    """Distinct arrival times e_0 < e_1 < ... inside [t_begin, t_end) and the per-event count of arriving
    spikes of every neuron, as (times, list of (neurons, counts))."""
    offs = np.asarray(offs, dtype=np.int64)
    times = np.asarray(times, dtype=np.float64)
    n = len(offs) - 1
    src = np.repeat(np.arange(n), np.diff(offs))
    arr = times + delay
    keep = arr < t_end
    arr, src = arr[keep], src[keep]
    order = np.argsort(arr, kind="stable")
    arr, src = arr[order], src[order]
    ev, first = np.unique(arr, return_index=True)
    groups = []
    for m in range(len(ev)):
        hi = first[m + 1] if m + 1 < len(ev) else len(arr)
        nj, cnt = np.unique(src[first[m]:hi], return_counts=True)
        groups.append((nj, cnt.astype(np.float64)))
    return ev, groups


def _interval_integral(u, a, D, tau):
    """tau (Ei(u) - Ei(u a)) elementwise (Eq. 10 for one interval), D where u = 0."""
    out = np.empty_like(u)
    z = u == 0.0
    nz = ~z
    out[nz] = tau * (expi(u[nz]) - expi(u[nz] * a[nz]))
    out[z] = D[z]
    return out


def _interval_weight(u, a, tau):
    """int_0^D exp(-s / tau) exp(u exp(-s / tau)) ds = tau (e^u - e^{u a}) / u (Eq. 14), tau (1 - a) at u = 0."""
    out = np.empty_like(u)
    z = u == 0.0
    nz = ~z
    out[nz] = tau * (np.exp(u[nz]) - np.exp(u[nz] * a[nz])) / u[nz]
    out[z] = tau * (1.0 - a[z])
    return out


def loglik_grad(offs, times, t_begin: float, t_end: float, tau: float, delay: float, W, b, *, grad: bool = True):
    """L_i, L, dL/dW, dL/db, dL/dtau of the continuous-time model (FP64).  Returns a dict with L (rows),
    L_total, G, gb, gtau_rows, gtau, C (the W-independent spike term sum_k v_j(t_ik)), q and the events."""
    offs = np.asarray(offs, dtype=np.int64)
    times = np.asarray(times, dtype=np.float64)
    W = np.asarray(W, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    n = len(offs) - 1
    ev, groups = arrival_events(offs, times, t_begin, t_end, delay)
    M = len(ev)
    # Eq. 8 / Eq. 13: u = U - b and v just after the arrivals at each event
    u_ev = np.zeros((n, M))
    v_ev = np.zeros((n, M))
    z_ev = np.zeros((n, M))  # z = W y (dL/dtau)
    u = np.zeros(n)
    v = np.zeros(n)
    z = np.zeros(n)
    t_prev = t_begin
    for m in range(M):
        gap = ev[m] - t_prev
        dec = np.exp(-gap / tau)
        z = dec * (z + gap * u)
        z_ev[:, m] = z
        u *= dec
        v *= dec
        nj, cnt = groups[m]
        u += W[:, nj] @ cnt
        v[nj] += cnt
        u_ev[:, m] = u
        v_ev[:, m] = v
        t_prev = ev[m]
    # intervals [t_begin, e_0) with u = 0, then [e_m, e_{m+1}) and [e_{M-1}, t_end)
    D0 = (ev[0] if M else t_end) - t_begin
    if M:
        D = np.diff(np.append(ev, t_end))
        a = np.exp(-D / tau)
        Da = np.broadcast_to(D, (n, M))
        aa = np.broadcast_to(a, (n, M))
        F = _interval_integral(u_ev, aa, Da, tau)
        integ = np.exp(b) * (D0 + F.sum(axis=1))
    else:
        integ = np.exp(b) * D0
    # spike part: U at each spike time from the last event at or before it
    q = np.diff(offs).astype(np.float64)
    Lsp = q * b
    C = np.zeros((n, n))
    zsp = np.zeros(n)  # sum over the row's spikes of z_i(t_ik)
    for i in range(n):
        ts = times[offs[i]:offs[i + 1]]
        if len(ts) == 0 or M == 0:
            continue
        ms = np.searchsorted(ev, ts, side="right") - 1
        ok = ms >= 0
        gap = ts[ok] - ev[ms[ok]]
        dec = np.exp(-gap / tau)
        Lsp[i] += np.dot(u_ev[i, ms[ok]], dec)
        zsp[i] = np.dot(z_ev[i, ms[ok]] + gap * u_ev[i, ms[ok]], dec)
        if grad:
            C[i] = v_ev[:, ms[ok]] @ dec
    L = Lsp - integ
    out = dict(L=L, L_total=float(L.sum()), q=q, events=ev, integ=integ)
    if grad:
        gint = np.zeros((n, n))
        gtau_rows = zsp / tau ** 2
        if M:
            Gw = _interval_weight(u_ev, aa, tau)
            gint = np.exp(b)[:, None] * (Gw @ v_ev.T)
            explicit = (F - Da * np.exp(u_ev * aa)) / tau  # (F - D e^{u a}) / tau, 0 where u = 0
            gtau_rows = gtau_rows - np.exp(b) * ((Gw * z_ev).sum(axis=1) / tau ** 2 + explicit.sum(axis=1))
        out.update(G=C - gint, gb=q - integ, C=C, gtau_rows=gtau_rows, gtau=float(gtau_rows.sum()))
    return out


def u_at(offs, times, t_begin: float, t_end: float, tau: float, delay: float, W, b, t_query):
    """U_i(t) for all rows at the given (sorted) times, by the recurrence (Eq. 8) and the decay to t."""
    W = np.asarray(W, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    ev, groups = arrival_events(offs, times, t_begin, t_end, delay)
    t_query = np.asarray(t_query, dtype=np.float64)
    out = np.empty((len(b), len(t_query)))
    u = np.zeros(len(b))
    t_prev = t_begin
    m = 0
    for k, t in enumerate(t_query):
        while m < len(ev) and ev[m] <= t:
            u *= np.exp(-(ev[m] - t_prev) / tau)
            nj, cnt = groups[m]
            u += W[:, nj] @ cnt
            t_prev = ev[m]
            m += 1
        out[:, k] = b + u * np.exp(-(t - t_prev) / tau)
    return out
