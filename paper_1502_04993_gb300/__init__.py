"""GB300 (sm_103a) maximum-likelihood reconstruction of recurrent synaptic connectivity from spike
trains with the point-process GLM of Zaytsev, Morrison & Deger.

Thin ctypes binding over ``libglm.so`` (C ABI in ``include/glm.h``).  Every step of the computation
runs in the library's CUDA kernels; this module only marshals arguments.  PyTorch supplies device
memory and streams.  There is no CPU fallback: importing the binding without the built library, or
using it without a CUDA device, raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libglm.so")

GLM_OK = 0
ERRORS = {
    -1: "GLM_ERR_INVALID_ARG", -2: "GLM_ERR_UNSORTED_SPIKES", -3: "GLM_ERR_SPIKE_OUT_OF_RANGE", -4: "GLM_ERR_OOM",
    -5: "GLM_ERR_CUDA", -6: "GLM_ERR_NONFINITE", -7: "GLM_ERR_TIMEOUT", -8: "GLM_ERR_UNSUPPORTED_ARCH",
    -9: "GLM_ERR_NO_PROBLEM", -10: "GLM_ERR_UNSUPPORTED",
}
PREC = {"f32": 0, "bf16": 1, "f16": 2}
DTYPE = {"f32": 0, "bf16": 1, "f16": 2}

# every symbol include/glm.h declares, with its ctypes signature
_vp, _i32, _i64, _f64, _sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
SIGNATURES = {
    "glm_version": ([], ctypes.c_int),
    "glm_strerror": ([ctypes.c_int], ctypes.c_char_p),
    "glm_last_error": ([_vp], ctypes.c_char_p),
    "glm_create": ([ctypes.POINTER(_vp), ctypes.c_int, _sz, _vp], ctypes.c_int),
    "glm_destroy": ([_vp], None),
    "glm_set_problem": ([_vp, _i32, _i64, _f64, _f64, _vp, _vp, ctypes.c_int], ctypes.c_int),
    "glm_prepare": ([_vp, _f64], ctypes.c_int),
    "glm_filter": ([_vp, _i64, _i64, _vp, _i64, ctypes.c_int], ctypes.c_int),
    "glm_spike_term": ([_vp, _vp, _vp], ctypes.c_int),
    "glm_loglik_grad": ([_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp], ctypes.c_int),
    "glm_profile_enable": ([_vp, ctypes.c_int], ctypes.c_int),
    "glm_profile_read": ([_vp, ctypes.c_int, _vp, _vp, _vp], ctypes.c_int),
    "glm_launch_count": ([_vp], _i64),
}



class ClassifyOpts(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int32), ("max_iter", ctypes.c_int32), ("tol", ctypes.c_double)]


class ClassifyReport(ctypes.Structure):
    _fields_ = [("centers", ctypes.c_double * 3), ("weights", ctypes.c_double * 3),
                ("variances", ctypes.c_double * 3), ("loglik", ctypes.c_double), ("iterations", ctypes.c_int32),
                ("errors", ctypes.c_int64), ("mer", ctypes.c_double), ("mer_n2", ctypes.c_double),
                ("fp", ctypes.c_int64 * 3), ("fn", ctypes.c_int64 * 3), ("nd", ctypes.c_int64 * 3)]


class FitOpts(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int32), ("m", ctypes.c_int32), ("max_iter", ctypes.c_int32),
                ("eta", ctypes.c_double), ("c1", ctypes.c_double), ("max_halvings", ctypes.c_int32),
                ("warm_start", ctypes.c_int32), ("gain_floor", ctypes.c_double), ("alpha", ctypes.c_double),
                ("eps", ctypes.c_double)]


class FitReport(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("evaluations", ctypes.c_int32), ("gradients", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("maxiter", ctypes.c_int32), ("stalled", ctypes.c_int32),
                ("degenerate", ctypes.c_int32), ("at_floor", ctypes.c_int32), ("excluded", ctypes.c_int32),
                ("L", ctypes.c_double),
                ("seconds", ctypes.c_double)]


class TuneReport(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("nsplit", ctypes.c_int32), ("cached", ctypes.c_int32),
                ("candidates", ctypes.c_int32), ("best_ms", ctypes.c_float)]


ROW_STATUS = {0: "converged", 1: "maxiter", 2: "stalled", 3: "degenerate", 4: "at_floor", 5: "excluded"}
ERRORS[-11] = "GLM_ERR_SCRATCH_TOO_SMALL"
SIGNATURES["glm_loglik_noalloc"] = ([_i32, _i64, _f64, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp], ctypes.c_int)
SIGNATURES["glm_fit_default_opts"] = ([ctypes.POINTER(FitOpts)], None)
SIGNATURES["glm_fit"] = ([_vp, ctypes.POINTER(FitOpts), _vp, _vp, _vp, ctypes.POINTER(FitReport)], ctypes.c_int)
SIGNATURES["glm_fit_batch"] = ([_vp, _i32, ctypes.POINTER(FitOpts), _vp, _vp, _vp, ctypes.POINTER(FitReport)], ctypes.c_int)
SIGNATURES["glm_autotune"] = ([_vp, _vp], ctypes.c_int)
SIGNATURES["glm_set_grad_tile"] = ([_vp, _i32, _i32, ctypes.POINTER(_i32)], ctypes.c_int)
SIGNATURES["glm_set_chunk_bins"] = ([_vp, _i64], ctypes.c_int)
SIGNATURES["glm_set_x_split"] = ([_vp, _i32], ctypes.c_int)
SIGNATURES["glm_set_source_delay"] = ([_vp, _i32], ctypes.c_int)
SIGNATURES["glm_set_self_delay"] = ([_vp, _i32], ctypes.c_int)
SIGNATURES["glm_set_row_range"] = ([_vp, _i32, _i32], ctypes.c_int)
SIGNATURES["glm_fit_classes"] = ([_vp, _i32, ctypes.POINTER(FitOpts), _vp, _vp, _vp, ctypes.POINTER(FitReport)],
                                 ctypes.c_int)
SIGNATURES["glm_ward"] = ([_vp, _vp, _i32, _i32, _vp, _i32, _vp], ctypes.c_int)
SIGNATURES["glm_ward_cut"] = ([_vp, _i32, _i32, _vp], ctypes.c_int)
SIGNATURES["glm_poison_caches"] = ([_vp], ctypes.c_int)
SIGNATURES["glm_check_wait_limit"] = ([_vp, _f64], ctypes.c_int)
SIGNATURES["glm_set_problem_ct"] = ([_vp, _i32, _f64, _f64, _f64, _f64, _vp, _vp, ctypes.c_int], ctypes.c_int)
SIGNATURES["glm_problem_columns"] = ([_vp, ctypes.POINTER(_i64)], ctypes.c_int)
SIGNATURES["glm_ct_interval"] = ([_f64, _f64, _f64, ctypes.POINTER(_f64), ctypes.POINTER(_f64)], ctypes.c_int)
SIGNATURES["glm_ct_interval_dtau"] = ([_f64, _f64, _f64, ctypes.POINTER(_f64)], ctypes.c_int)
SIGNATURES["glm_expm1"] = ([_vp, _i64, _vp], ctypes.c_int)
SIGNATURES["glm_cross_validate"] = ([_vp, _vp, ctypes.POINTER(FitOpts), _vp, _i32, _vp, _i32, _vp, _vp, _vp, _vp],
                                     ctypes.c_int)
SIGNATURES["glm_classify"] =([_vp, _i32, ctypes.POINTER(ClassifyOpts), _vp, _vp, _vp, ctypes.POINTER(ClassifyReport)],
                              ctypes.c_int)

# precisions the library implements
AVAILABLE_PRECISIONS = ("f32", "bf16", "f16")


def available_precisions():
    return AVAILABLE_PRECISIONS

_lib = None


class GLMError(RuntimeError):
    def __init__(self, code: int, msg: str = ""):
        self.code = code
        super().__init__(f"{ERRORS.get(code, code)}: {msg}" if msg else f"{ERRORS.get(code, code)}")


def load_library(path: str = LIB_PATH):
    """Load libglm.so and declare its signatures.  Raises if the library was not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libglm.so not found at {path}: build it first (python -m paper_1502_04993_gb300.build "
                          "or __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    for name, (args, res) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _ptr(t) -> int | None:
    return None if t is None else t.data_ptr()


def fit_batch(contexts, *, method: str = "lbfgs", m: int = 10, max_iter: int = 500, eta: float = 1e-10,
              c1: float = 1e-4, max_halvings: int = 40, gain_floor: float = -1.0, alpha: float = 0.0,
              eps: float = 1e-6):
    """Fit the problems of several contexts together (glm_fit_batch): one launch per contraction over all
    problems, one CUDA graph per optimiser iteration.  Returns a list of dict(W, b, status, report), one per
    context, and the call's status code."""
    lib = load_library()
    k = len(contexts)
    if k == 0:
        raise ValueError("no contexts")
    torch = contexts[0].torch
    Ws, bs, sts = [], [], []
    for g in contexts:
        dev = f"cuda:{g.device}"
        Ws.append(torch.zeros((g.n, g.n), dtype=torch.float32, device=dev))
        bs.append(torch.zeros(g.n, dtype=torch.float32, device=dev))
        sts.append(np.zeros(g.n, dtype=np.int8))
    arr = ctypes.c_void_p * k
    hs = arr(*[g.h for g in contexts])
    wp = arr(*[w.data_ptr() for w in Ws])
    bp = arr(*[b.data_ptr() for b in bs])
    sp = arr(*[s.ctypes.data for s in sts])
    reps = (FitReport * k)()
    o = FitOpts({"lbfgs": 0, "ga": 1}[method], m, max_iter, eta, c1, max_halvings, 0, gain_floor, alpha, eps)
    rc = lib.glm_fit_batch(hs, k, ctypes.byref(o), wp, bp, sp, reps)
    if rc < 0:
        contexts[0]._check(rc, "glm_fit_batch")
    out = [dict(W=Ws[p], b=bs[p], status=sts[p], report={f: getattr(reps[p], f) for f, _ in FitReport._fields_})
           for p in range(k)]
    return out, rc


def fit_classes(contexts, W=None, b=None, *, method: str = "lbfgs", m: int = 10, max_iter: int = 500,
                eta: float = 1e-10, c1: float = 1e-4, max_halvings: int = 40, gain_floor: float = -1.0,
                alpha: float = 0.0, eps: float = 1e-6):
    """Fit the row classes held by several contexts (glm_fit_classes): each context has its own tau, source
    delay and row range, and all of them write into one W (n x n) and b (n).  W and b, when given, are the
    warm start (and the values kept for rows in no range).  Returns dict(W, b, status, report, rc)."""
    lib = load_library()
    k = len(contexts)
    if k == 0:
        raise ValueError("no contexts")
    g0 = contexts[0]
    torch = g0.torch
    dev = f"cuda:{g0.device}"
    warm = W is not None
    Wd = (W.to(device=dev, dtype=torch.float32).clone() if warm
          else torch.zeros((g0.n, g0.n), dtype=torch.float32, device=dev)).contiguous()
    bd = (b.to(device=dev, dtype=torch.float32).clone() if warm
          else torch.zeros(g0.n, dtype=torch.float32, device=dev)).contiguous()
    status = np.zeros(g0.n, dtype=np.int8)
    hs = (ctypes.c_void_p * k)(*[g.h for g in contexts])
    o = FitOpts({"lbfgs": 0, "ga": 1}[method], m, max_iter, eta, c1, max_halvings, int(warm), gain_floor, alpha,
                eps)
    rep_ = FitReport()
    rc = lib.glm_fit_classes(hs, k, ctypes.byref(o), _ptr(Wd), _ptr(bd), status.ctypes.data, ctypes.byref(rep_))
    if rc < 0:
        g0._check(rc, "glm_fit_classes")
    return dict(W=Wd, b=bd, status=status, report={f: getattr(rep_, f) for f, _ in FitReport._fields_}, rc=rc)


def ward_cut(Z, k: int) -> np.ndarray:
    """Labels of the k clusters of a linkage (glm_ward_cut)."""
    lib = load_library()
    Z = np.ascontiguousarray(Z, dtype=np.float64)
    m = Z.shape[0] + 1
    lab = np.zeros(m, dtype=np.int32)
    rc = lib.glm_ward_cut(Z.ctypes.data, m, int(k), lab.ctypes.data)
    if rc != GLM_OK:
        raise GLMError(rc, "glm_ward_cut")
    return lab


def expm1(v) -> np.ndarray:
    """e^v - 1 of float32 values as the plain FP32 form's epilogue computes it (host code of libglm)."""
    lib = load_library()
    v = np.ascontiguousarray(v, dtype=np.float32)
    out = np.empty_like(v)
    rc = lib.glm_expm1(v.ctypes.data, v.size, out.ctypes.data)
    if rc != GLM_OK:
        raise GLMError(rc, "glm_expm1")
    return out


def ct_interval(u: float, D: float, tau: float):
    """(F, G) of one continuous-time column (glm_ct_interval; host code, no GPU needed)."""
    lib = load_library()
    F, G = ctypes.c_double(), ctypes.c_double()
    rc = lib.glm_ct_interval(float(u), float(D), float(tau), ctypes.byref(F), ctypes.byref(G))
    if rc != GLM_OK:
        raise GLMError(rc, "glm_ct_interval")
    return F.value, G.value


def ct_interval_dtau(u: float, D: float, tau: float) -> float:
    """dF/dtau at fixed u of one continuous-time column (glm_ct_interval_dtau; host code, no GPU needed)."""
    lib = load_library()
    out = ctypes.c_double()
    rc = lib.glm_ct_interval_dtau(float(u), float(D), float(tau), ctypes.byref(out))
    if rc != GLM_OK:
        raise GLMError(rc, "glm_ct_interval_dtau")
    return out.value


def split_recording(offs, bins, n_bins: int, t_split: int):
    """Split a CSR recording at bin t_split into a training part [0, t_split) and a validation part
    [t_split, n_bins) whose bins are counted from t_split (for glm_cross_validate).  Returns
    ((offs, bins, t_split), (offs, bins, n_bins - t_split))."""
    offs = np.ascontiguousarray(offs, dtype=np.int64)
    bins = np.ascontiguousarray(bins, dtype=np.int32)
    if not 0 < t_split < n_bins:
        raise ValueError("t_split must lie inside the recording")
    n = offs.size - 1
    rows = np.repeat(np.arange(n), np.diff(offs))
    early = bins < t_split
    parts = []
    for keep, base, length in ((early, 0, t_split), (~early, t_split, n_bins - t_split)):
        o = np.zeros(n + 1, dtype=np.int64)
        np.cumsum(np.bincount(rows[keep], minlength=n), out=o[1:])
        parts.append((o, (bins[keep] - base).astype(np.int32), int(length)))
    return tuple(parts)


def split_recording_ct(offs, times, t_begin: float, t_end: float, t_split: float):
    """Split a continuous-time recording at t_split into a training window [t_begin, t_split) and a
    validation window [t_split, t_end), times kept as they are.  Returns
    ((offs, times, t_begin, t_split), (offs, times, t_split, t_end))."""
    offs = np.ascontiguousarray(offs, dtype=np.int64)
    times = np.ascontiguousarray(times, dtype=np.float64)
    if not t_begin < t_split < t_end:
        raise ValueError("t_split must lie inside the recording")
    n = offs.size - 1
    rows = np.repeat(np.arange(n), np.diff(offs))
    early = times < t_split
    parts = []
    for keep, lo, hi in ((early, t_begin, t_split), (~early, t_split, t_end)):
        o = np.zeros(n + 1, dtype=np.int64)
        o[1:] = np.cumsum(np.bincount(rows[keep], minlength=n))
        parts.append((o, times[keep].copy(), lo, hi))
    return parts[0], parts[1]


def cross_validate(train, valid, alphas, taus=None, **fit_kw):
    """glm_cross_validate: fit on context `train` for every alpha (and tau), score on context `valid`.
    Returns dict(L_valid [n_tau x n_alpha], best (k_tau, k_alpha), W, b at the best point)."""
    lib = load_library()
    torch = train.torch
    alphas = np.ascontiguousarray(alphas, dtype=np.float64)
    tau_arr = None if taus is None else np.ascontiguousarray(taus, dtype=np.float64)
    n_tau = 1 if tau_arr is None else tau_arr.size
    L = np.zeros((n_tau, alphas.size))
    best = np.zeros(2, dtype=np.int32)
    dev = f"cuda:{train.device}"
    W = torch.zeros((train.n, train.n), dtype=torch.float32, device=dev)
    b = torch.zeros(train.n, dtype=torch.float32, device=dev)
    kw = dict(method="lbfgs", m=10, max_iter=500, eta=1e-10, c1=1e-4, max_halvings=40, gain_floor=-1.0, eps=1e-6)
    kw.update(fit_kw)
    o = FitOpts({"lbfgs": 0, "ga": 1}[kw["method"]], kw["m"], kw["max_iter"], kw["eta"], kw["c1"],
                kw["max_halvings"], 0, kw["gain_floor"], 0.0, kw["eps"])
    rc = lib.glm_cross_validate(train.h, valid.h, ctypes.byref(o), alphas.ctypes.data, alphas.size,
                                None if tau_arr is None else tau_arr.ctypes.data, n_tau, L.ctypes.data,
                                best.ctypes.data, _ptr(W), _ptr(b))
    train._check(rc, "glm_cross_validate")
    return dict(L_valid=L, best=(int(best[0]), int(best[1])), W=W, b=b)


def classify(W, method: str = "gmm", truth=None, types=None, max_iter: int = 1000, tol: float = 1e-12):
    """Labels (n x n int8: -1 inhibitory, 0 absent, +1 excitatory) of the off-diagonal weights and a report
    dict (cluster centres, and with `truth` the misclassification rate and its FP/FN/ND breakdown).
    Host computation in libglm (glm_classify)."""
    lib = load_library()
    W = np.ascontiguousarray(W, dtype=np.float64)
    n = W.shape[0]
    labels = np.zeros((n, n), dtype=np.int8)
    tr = None if truth is None else np.ascontiguousarray(truth, dtype=np.int8)
    ty = None if types is None else np.ascontiguousarray(types, dtype=np.int8)
    o = ClassifyOpts({"gmm": 0, "kmeans": 1}[method], max_iter, tol)
    rep = ClassifyReport()
    rc = lib.glm_classify(W.ctypes.data, n, ctypes.byref(o), labels.ctypes.data,
                          None if tr is None else tr.ctypes.data, None if ty is None else ty.ctypes.data,
                          ctypes.byref(rep))
    if rc != GLM_OK:
        raise GLMError(rc, "glm_classify")
    names = ("inh", "absent", "exc")
    out = dict(centers=list(rep.centers), weights=list(rep.weights), variances=list(rep.variances),
               loglik=rep.loglik, iterations=rep.iterations)
    if tr is not None:
        out.update(errors=rep.errors, mer=rep.mer, mer_n2=rep.mer_n2)
        for k, nm in enumerate(names):
            out[nm] = dict(errors=rep.fp[k] + rep.fn[k], fp=rep.fp[k], fn=rep.fn[k], nd=rep.nd[k])
    return labels, out


class GLM:
    """One libglm context on one CUDA device, bound to a torch stream."""

    def __init__(self, device: int = 0, workspace_cap: int = 0, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libglm needs a CUDA device; there is no CPU fallback")
        self.lib = load_library()
        self.device = device
        self.torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        h = ctypes.c_void_p()
        rc = self.lib.glm_create(ctypes.byref(h), device, workspace_cap, ctypes.c_void_p(self.stream.cuda_stream))
        if rc != GLM_OK:
            raise GLMError(rc, "glm_create")
        self.h = h
        self.n = self.n_bins = None

    # ---- helpers ----
    def _check(self, rc: int, what: str):
        if rc != GLM_OK:
            msg = self.lib.glm_last_error(self.h)
            raise GLMError(rc, f"{what}: {msg.decode() if msg else ''}")
        return rc

    def close(self):
        if getattr(self, "h", None):
            self.lib.glm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- API ----
    def set_problem(self, offs, bins, n_bins: int, dt: float, tau: float, prec: str = "f32"):
        offs = np.ascontiguousarray(offs, dtype=np.int64)
        bins = np.ascontiguousarray(bins, dtype=np.int32)
        n = offs.size - 1
        rc = self.lib.glm_set_problem(self.h, n, int(n_bins), float(dt), float(tau), offs.ctypes.data,
                                      bins.ctypes.data if bins.size else None, PREC[prec])
        self._check(rc, "glm_set_problem")
        self.n, self.n_bins, self.dt, self.tau, self.prec = n, int(n_bins), dt, tau, prec

    def set_problem_ct(self, offs, times, t_begin: float, t_end: float, tau: float, delay: float,
                       prec: str = "bf16"):
        """Continuous-time problem (glm_set_problem_ct): spike times in seconds, one uniform delay."""
        offs = np.ascontiguousarray(offs, dtype=np.int64)
        times = np.ascontiguousarray(times, dtype=np.float64)
        n = offs.size - 1
        rc = self.lib.glm_set_problem_ct(self.h, n, float(t_begin), float(t_end), float(tau), float(delay),
                                         offs.ctypes.data, times.ctypes.data if times.size else None, PREC[prec])
        self._check(rc, "glm_set_problem_ct")
        self.n, self.tau, self.prec = n, tau, prec
        self.n_bins, self.dt = self.columns(), None

    def set_source_delay(self, delay_bins: int):
        """Delay of the source trains in bins (>= 1), applied at the next set_problem (glm_set_source_delay)."""
        self._check(self.lib.glm_set_source_delay(self.h, int(delay_bins)), "glm_set_source_delay")

    def set_self_delay(self, self_bins: int):
        """Each row's own train reaches it after self_bins bins, the others after the source delay
        (glm_set_self_delay; applies at the next set_problem)."""
        self._check(self.lib.glm_set_self_delay(self.h, int(self_bins)), "glm_set_self_delay")

    def set_row_range(self, r0: int, r1: int):
        """Evaluate and fit rows [r0, r1) only (glm_set_row_range); (0, 0) restores all rows."""
        self._check(self.lib.glm_set_row_range(self.h, int(r0), int(r1)), "glm_set_row_range")

    def ward(self, W, by: str = "out", subset=None) -> np.ndarray:
        """Ward linkage of neurons by their outgoing (by='out') or incoming ('in') weights (glm_ward)."""
        torch = self.torch
        Wd = W.to(device=f"cuda:{self.device}", dtype=torch.float32).contiguous()
        n = Wd.shape[0]
        sub = None if subset is None else np.ascontiguousarray(subset, dtype=np.int32)
        m = n if sub is None else sub.size
        Z = np.zeros((max(m - 1, 0), 4), dtype=np.float64)
        rc = self.lib.glm_ward(self.h, _ptr(Wd), n, {"out": 0, "in": 1}[by], None if sub is None else sub.ctypes.data,
                               m, Z.ctypes.data)
        self._check(rc, "glm_ward")
        return Z

    def poison_caches(self):
        """Fill every recomputed buffer with NaN bytes (glm_poison_caches); glm_prepare restores them."""
        self._check(self.lib.glm_poison_caches(self.h), "glm_poison_caches")

    def check_wait_limit(self, limit_seconds: float = 0.05) -> int:
        """Status of a bounded wait that nobody satisfies (glm_check_wait_limit): GLM_ERR_TIMEOUT expected."""
        return int(self.lib.glm_check_wait_limit(self.h, float(limit_seconds)))

    def columns(self) -> int:
        """Time columns of the current problem (bins, or event columns in continuous time)."""
        m = ctypes.c_int64()
        self._check(self.lib.glm_problem_columns(self.h, ctypes.byref(m)), "glm_problem_columns")
        return int(m.value)

    def prepare(self, tau: float | None = None):
        self._check(self.lib.glm_prepare(self.h, float(tau) if tau else -1.0), "glm_prepare")
        if tau:
            self.tau = tau

    def filter(self, t0: int = 0, t_len: int | None = None, dtype: str = "f32", out=None):
        torch = self.torch
        t_len = self.n_bins - t0 if t_len is None else t_len
        tdt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[dtype]
        if out is None:
            out = torch.empty((self.n, t_len), dtype=tdt, device=f"cuda:{self.device}")
        self._check(self.lib.glm_filter(self.h, int(t0), int(t_len), _ptr(out), out.stride(0), DTYPE[dtype]),
                    "glm_filter")
        return out

    def spike_term(self):
        torch = self.torch
        C = torch.empty((self.n, self.n), dtype=torch.float64, device=f"cuda:{self.device}")
        q = torch.empty(self.n, dtype=torch.float64, device=f"cuda:{self.device}")
        self._check(self.lib.glm_spike_term(self.h, _ptr(C), _ptr(q)), "glm_spike_term")
        return C, q

    def profile(self, enable: bool = True):
        self._check(self.lib.glm_profile_enable(self.h, int(enable)), "glm_profile_enable")

    def profile_read(self) -> dict:
        """{group name: (launches, total ms)} since profiling was enabled (synchronises)."""
        m = 16
        names = ctypes.create_string_buffer(32 * m)
        cnt = (ctypes.c_int64 * m)()
        ms = (ctypes.c_double * m)()
        k = self.lib.glm_profile_read(self.h, m, names, cnt, ms)
        if k < 0:
            raise GLMError(k, "glm_profile_read")
        raw = names.raw
        out = {}
        for e in range(k):
            nm = raw[32 * e:32 * e + 32].split(b"\0", 1)[0].decode()
            out[nm] = (int(cnt[e]), float(ms[e]))
        return out

    def launch_count(self) -> int:
        return int(self.lib.glm_launch_count(self.h))

    def fit(self, W=None, b=None, *, method: str = "lbfgs", m: int = 10, max_iter: int = 500, eta: float = 1e-10,
            c1: float = 1e-4, max_halvings: int = 40, gain_floor: float = -1.0, alpha: float = 0.0,
            eps: float = 1e-6):
        """Maximum-likelihood W, b of the current problem (glm_fit).  Starts at W = 0, b = log(q / T dt) unless
        W and b are given (warm start).  Returns dict(W, b, status per row, report, rc)."""
        torch = self.torch
        dev = f"cuda:{self.device}"
        warm = W is not None
        Wd = (W.to(device=dev, dtype=torch.float32).clone() if warm
              else torch.zeros((self.n, self.n), dtype=torch.float32, device=dev)).contiguous()
        bd = (b.to(device=dev, dtype=torch.float32).clone() if warm
              else torch.zeros(self.n, dtype=torch.float32, device=dev)).contiguous()
        o = FitOpts({"lbfgs": 0, "ga": 1}[method], m, max_iter, eta, c1, max_halvings, int(warm), gain_floor, alpha,
                    eps)
        rep = FitReport()
        status = np.zeros(self.n, dtype=np.int8)
        rc = self.lib.glm_fit(self.h, ctypes.byref(o), _ptr(Wd), _ptr(bd), status.ctypes.data, ctypes.byref(rep))
        if rc < 0:
            self._check(rc, "glm_fit")
        report = {f: getattr(rep, f) for f, _ in FitReport._fields_}
        return dict(W=Wd, b=bd, status=status, report=report, rc=rc)

    def set_chunk_bins(self, chunk_bins: int):
        """Recompute X in chunks of this many bins instead of storing it (applies to the next set_problem)."""
        self._check(self.lib.glm_set_chunk_bins(self.h, int(chunk_bins)), "glm_set_chunk_bins")

    def set_x_split(self, split: bool):
        """16-bit grid forms: hold X as X_hi + X_lo (True, default) or as one 16-bit X (False); applies to
        the next set_problem (glm_set_x_split)."""
        self._check(self.lib.glm_set_x_split(self.h, int(bool(split))), "glm_set_x_split")

    def set_grad_tile(self, mode: int, units_per_sm: int) -> int:
        """Force one of the autotuner's gradient-product tile shapes; returns the resulting bin splits."""
        ns = ctypes.c_int32(0)
        self._check(self.lib.glm_set_grad_tile(self.h, int(mode), int(units_per_sm), ctypes.byref(ns)),
                    "glm_set_grad_tile")
        return ns.value

    def autotune(self) -> dict:
        """Time the gradient product's tile shapes for this problem and keep the fastest (glm_autotune)."""
        rep = TuneReport()
        self._check(self.lib.glm_autotune(self.h, ctypes.byref(rep)), "glm_autotune")
        return {f: getattr(rep, f) for f, _ in TuneReport._fields_}

    def loglik_grad(self, W, b, *, grad: bool = True, total: bool = True, tau_grad: bool = False, out=None):
        """L_i, L, dL/dW, dL/db (and with tau_grad dL/dtau) at (W, b).  W: (n, n) float32, b: (n,) float32."""
        torch = self.torch
        dev = f"cuda:{self.device}"
        W = W.to(device=dev, dtype=torch.float32).contiguous()
        b = b.to(device=dev, dtype=torch.float32).contiguous()
        if self.n is None:  # no problem yet: let the library report it
            self._check(self.lib.glm_loglik_grad(self.h, _ptr(W), _ptr(b), None, None, None, None, None),
                        "glm_loglik_grad")
        out = out or {}
        L_rows = out.get("L_rows")
        if L_rows is None:
            L_rows = torch.empty(self.n, dtype=torch.float64, device=dev)
        G = out.get("G") if grad else None
        if grad and G is None:
            G = torch.empty((self.n, self.n), dtype=torch.float64, device=dev)
        gb = out.get("gb") if grad else None
        if grad and gb is None:
            gb = torch.empty(self.n, dtype=torch.float64, device=dev)
        tot = ctypes.c_double(0.0)
        gt = ctypes.c_double(0.0)
        rc = self.lib.glm_loglik_grad(self.h, _ptr(W), _ptr(b), _ptr(L_rows),
                                      ctypes.byref(tot) if total else None, _ptr(G), _ptr(gb),
                                      ctypes.byref(gt) if tau_grad else None)
        self._check(rc, "glm_loglik_grad")
        return dict(L_rows=L_rows, L_total=tot.value if total else None, G=G, gb=gb,
                    gtau=gt.value if tau_grad else None)
