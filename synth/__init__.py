"""Seeded synthetic spike data for the GLM reconstruction path.

Builds the random balanced E/I networks and the spike rasters that stand in
for the paper's simulated recordings (Sec. 3.1: N neurons, 80:20 E:I, random
connections with probability p, a few Hz, hour-scale recordings).  The spike
trains are simulated from the discrete-time model itself (Eq. 3-5 on a grid
with a one-bin delay, Eq. 8 as the potential recursion), Bernoulli per bin
with the rate capped at 200 Hz.

This module makes inputs only.  It shares no code with either the FP64 oracle
or the CUDA library and holds none of their evaluation arithmetic; both sides
receive its CSR spike trains (``offs``, ``bins``) as plain arrays.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "glm_synth.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libglm_synth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the generator with gcc (OpenMP, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u32p = ctypes.POINTER(ctypes.c_uint32)
            lib.synth_philox4x32_10.argtypes = [u32p, u32p, u32p]
            lib.synth_philox4x32_10.restype = None
            lib.synth_network.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_double, ctypes.c_int32, ctypes.c_uint64, ctypes.c_void_p,
                                          ctypes.c_void_p]
            lib.synth_network.restype = ctypes.c_int
            lib.synth_simulate.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_uint64,
                                           ctypes.c_int32]
            lib.synth_simulate.restype = ctypes.c_void_p
            lib.synth_sim_count.argtypes = [ctypes.c_void_p]
            lib.synth_sim_count.restype = ctypes.c_int64
            lib.synth_sim_copy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            lib.synth_sim_copy.restype = None
            lib.synth_sim_free.argtypes = [ctypes.c_void_p]
            lib.synth_sim_free.restype = None
            _lib = lib
    return _lib


def philox4x32_10(ctr, key) -> tuple:
    """One Philox4x32-10 block: 4 counter words, 2 key words -> 4 output words."""
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib.synth_philox4x32_10(c, k, o)
    return tuple(int(x) for x in o)


def network(n: int, n_exc: int, p: float, w_exc: float, w_inh: float, seed: int, *, w_self: float = 0.0,
            syn_groups: int = 0, syn_size: int = 0, w_syn: float = 0.0, shuffle: bool = False):
    """Random network: W[i, j] is the weight of j -> i (+w_exc from E, -w_inh from I); diagonal = w_self."""
    lib = _load()
    W = np.zeros((n, n), dtype=np.float64)
    types = np.zeros(n, dtype=np.int8)
    rc = lib.synth_network(n, n_exc, p, w_exc, w_inh, w_self, syn_groups, syn_size, w_syn, int(shuffle), seed,
                           W.ctypes.data, types.ctypes.data)
    if rc != 0:
        raise ValueError(f"synth_network failed ({rc})")
    return W, types


def simulate(W: np.ndarray, b: np.ndarray, tau: float, dt: float, n_bins: int, seed: int, *,
             rate_cap: float = 200.0, threads: int = 0):
    """Simulate the grid GLM; returns CSR spike trains (offs int64[n+1], bins int32[q], sorted per row)."""
    lib = _load()
    W = np.ascontiguousarray(W, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    n = W.shape[0]
    h = lib.synth_simulate(n, int(n_bins), float(dt), float(tau), W.ctypes.data, b.ctypes.data,
                           float(rate_cap), int(seed), int(threads))
    if not h:
        raise ValueError("synth_simulate failed")
    try:
        q = lib.synth_sim_count(h)
        offs = np.zeros(n + 1, dtype=np.int64)
        bins = np.zeros(max(q, 1), dtype=np.int32)
        lib.synth_sim_copy(h, offs.ctypes.data, bins.ctypes.data)
    finally:
        lib.synth_sim_free(h)
    return offs, bins[:q]


# Named workloads.  Shapes follow the paper's balanced GLM network experiment
# (Sec. 3.1 and App. C.3: 80:20 E:I, p = 0.1, a few Hz, hour-scale recordings)
# scaled to a 1 ms grid.
WORKLOADS = {
    # N=50 (40 E / 10 I), 20 s: the small case the FP64 oracle fits in seconds
    "glm_n50_t20k": dict(n=50, n_exc=40, p=0.1, w_exc=0.5, w_inh=2.0, rate=5.0, tau=0.010, dt=0.001,
                         n_bins=20_000, seed=0),
    # N=1000 (800 E / 200 I), 1800 s on a 1 ms grid (1.8M bins).  The refractory self-connection
    # -6.25 is the paper's J_s = -25 mV at du = 4 mV (Sec. 3.1); without it this network leaves the
    # low-rate state and settles near 80 Hz.
    "glm_n1000_t1800s": dict(n=1000, n_exc=800, p=0.1, w_exc=0.2, w_inh=0.8, w_self=-6.25, rate=8.0,
                             tau=0.010, dt=0.001, n_bins=1_800_000, seed=0),
    # N=2000 (1600 E / 400 I) with a 10 x 50 synfire chain, 3600 s.  In this exponential-rate model the
    # +0.3 chain drives the network into saturation (mean rate 97 Hz) unless each chain neuron's baseline
    # is lowered; syn_b_comp = 2 lowers it by twice its expected input from the previous link,
    # 50 x 0.3 x rate x tau (mean rate then 5.2 Hz: chain neurons 1.5 Hz, background 6.5 Hz).
    "glm_n2000_synfire_t3600s": dict(n=2000, n_exc=1600, p=0.05, w_exc=0.2, w_inh=0.8, w_self=-6.25,
                                     rate=8.0, tau=0.010, dt=0.001, n_bins=3_600_000, seed=0, syn_groups=10,
                                     syn_size=50, w_syn=0.3, shuffle=True, syn_b_comp=2.0),
}


def truth_labels(W_true: np.ndarray) -> np.ndarray:
    """Ground-truth connection classes of a generated network: +1 excitatory, -1 inhibitory, 0 absent
    (W_true[i, j] is the weight from j onto i; the diagonal, the self-coupling, is no connection)."""
    W_true = np.asarray(W_true)
    lab = np.sign(W_true).astype(np.int8)
    np.fill_diagonal(lab, 0)
    return lab


def make_workload(name: str | None = None, *, threads: int = 0, **overrides) -> dict:
    """Generate a named workload (ground truth + spikes).  Any field may be overridden."""
    cfg = dict(WORKLOADS[name]) if name else {}
    cfg.update(overrides)
    W, types = network(cfg["n"], cfg["n_exc"], cfg["p"], cfg["w_exc"], cfg["w_inh"], cfg["seed"],
                       w_self=cfg.get("w_self", 0.0), syn_groups=cfg.get("syn_groups", 0),
                       syn_size=cfg.get("syn_size", 0), w_syn=cfg.get("w_syn", 0.0),
                       shuffle=cfg.get("shuffle", False))
    b = np.full(cfg["n"], math.log(cfg["rate"]), dtype=np.float64)
    if cfg.get("syn_groups", 0) and cfg.get("syn_b_comp", 0.0):
        # chain neurons: baseline lowered by syn_b_comp x their expected input from the previous link
        w_syn = cfg["w_syn"]
        n_in = np.isclose(W, w_syn).sum(axis=1)
        b -= cfg["syn_b_comp"] * n_in * w_syn * cfg["rate"] * cfg["tau"]
    offs, bins = simulate(W, b, cfg["tau"], cfg["dt"], cfg["n_bins"], cfg["seed"], threads=threads)
    out = dict(cfg)
    out.update(W_true=W, b_true=b, types=types, offs=offs, bins=bins)
    return out


def batch_workloads(n_rec: int = 24, *, scale: float = 1.0, t_scale: float | None = None):
    """Uneven recordings for batched fitting: N ~ U{100..1500}, T ~ U(300, 3600) s, rate ~ U(3, 12) Hz,
    80/20 E/I, p = 0.1, +0.2 / -0.8, seeds 1..n_rec.  ``scale`` shrinks N and T for tests; ``t_scale``, when
    given, shrinks T alone."""
    out = []
    for s in range(1, n_rec + 1):
        w = philox4x32_10((s, 0, 0, 0x42415443), (s, 0))
        n = max(8, int(round((100 + w[0] % 1401) * scale)))
        t_sec = 300.0 + (w[1] / 4294967296.0) * 3300.0
        rate = 3.0 + (w[2] / 4294967296.0) * 9.0
        n_bins = max(64, int(round(t_sec * 1000 * (scale if t_scale is None else t_scale))))
        out.append(dict(n=n, n_exc=int(round(0.8 * n)), p=0.1, w_exc=0.2, w_inh=0.8, w_self=-6.25, rate=rate,
                        tau=0.010, dt=0.001, n_bins=n_bins, seed=s))
    return out


def continuous_times(offs, bins, dt: float, seed: int) -> np.ndarray:
    """Off-grid spike times for the continuous-time form: spike k at (bins[k] + u_k) dt with u_k uniform in
    [0, 1) from a Philox stream keyed by ``seed``.  Rows stay strictly increasing (one spike per bin)."""
    bins = np.asarray(bins, dtype=np.int64)
    u = np.random.Generator(np.random.Philox(key=int(seed))).random(len(bins))
    return (bins.astype(np.float64) + u) * dt


def make_ct_workload(name: str | None = None, *, jitter_seed: int = 7, delay: float | None = None,
                     threads: int = 0, **overrides) -> dict:
    """A grid workload (``make_workload``) with its spikes moved off the grid (``continuous_times``), on the
    recording window [0, n_bins dt).  ``delay`` (default one bin, dt) is the uniform transmission delay."""
    w = make_workload(name, threads=threads, **overrides)
    w["times"] = continuous_times(w["offs"], w["bins"], w["dt"], jitter_seed)
    w["t_begin"] = 0.0
    w["t_end"] = w["n_bins"] * w["dt"]
    w["delay"] = w["dt"] if delay is None else float(delay)
    return w
