#!/usr/bin/env python
"""Benchmark of the GLM log-likelihood + gradient hot path: neuron*bins/s on the N = 1000 neuron,
1800 s (1.8M bins of 1 ms) balanced-network workload.

One step = the whole hot path once: filter scan and spike term from the device-resident spikes
(steps a0-a2), then U = b + W X with the fused link epilogue, the gradient product and the FP64
reductions (a3-a5, a7).  `value` times K such steps with the inputs already in HBM; `e2e` times the
same through the public API from host buffers (spike upload and validation, W/b upload, L and G read
back).  The default form holds X as one FP16 array and W as an FP16 hi + lo pair (--prec f16x1); f16 and
bf16 hold X as X_hi + X_lo, bf16x1 as one BF16 array, f32 is the plain FP32 form.  After the timed steps,
untimed legs add to the same line: the full fit in the default form and in the plain FP32 form (wall time,
iterations, misclassification rate, speed-up over FP32), the continuous-time
form on the first 180 s, the recording as four row classes with their own tau and delay, and the FP64
oracle on a bounded sample of the host cores.  Prints one JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--prec f16x1|f16|bf16|bf16x1|f32] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "glm_n1000_t1800s"
METRIC = "GLM loglik+grad neuron*bins/s at N=1000"
UNIT = "neuron*bins/s"
# evaluation forms: name -> (precision of the contractions, X held as X_hi + X_lo)
FORMS = {"f16x1": ("f16", False), "bf16x1": ("bf16", False), "f16": ("f16", True), "bf16": ("bf16", True),
         "f32": ("f32", True)}
DEFAULT_FORM = "f16x1"


def use_form(ctx, form: str) -> str:
    """Set the context's X split for the form (applies at its next set_problem); returns the precision."""
    prec, split = FORMS[form]
    ctx.set_x_split(split)
    return prec


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default=None, choices=sorted(FORMS),
                    help=f"evaluation form (default {DEFAULT_FORM}: FP16 contractions, one FP16 X, W as hi + lo)")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--n-bins", type=int, default=None,
                    help="record a shorter recording of the same network (profiling captures)")
    ap.add_argument("--fit", default=f"{DEFAULT_FORM},f32",
                    help="comma list of forms to also run the full glm_fit with, reporting wall time, the "
                         "misclassification rate and the speed-up over the plain FP32 form ('' : off); with f32 "
                         "in the list, the first other form is also finished by the FP32 form from its result")
    ap.add_argument("--fit-eta", type=float, default=1e-9)
    ap.add_argument("--fit-max-iter", type=int, default=400)
    ap.add_argument("--batch", type=int, default=0,
                    help="also fit this many uneven recordings with glm_fit_batch and one after another")
    ap.add_argument("--batch-t-scale", type=float, default=0.1, help="recording-length scale of --batch")
    ap.add_argument("--ct-seconds", type=float, default=180.0,
                    help="also evaluate and fit the continuous-time form on this much of the recording, its spikes "
                         "moved off the grid (0: off)")
    ap.add_argument("--no-ct-fit", action="store_true", help="continuous-time leg without its fits (profiling)")
    ap.add_argument("--classes", type=int, default=4,
                    help="also evaluate the recording as this many row classes with their own tau and delay (0: off)")
    ap.add_argument("--undersampling", default="",
                    help="comma list of sampled fractions (e.g. 0.25,0.5,0.75,1): refit on random neuron subsets "
                         "with the E:I ratio kept and report the misclassification rate (k-means and GMM)")
    ap.add_argument("--synfire", action="store_true",
                    help="also fit the N = 2000 synfire-chain recording and find its links by Ward clustering")
    ap.add_argument("--synfire-seconds", type=float, default=3600.0)
    return ap.parse_args()


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_seed(base_seed: int, rank: int) -> int:
    """Seed of rank `rank`'s recording: every GPU fits its own independent recording (weak scaling)."""
    return base_seed + rank


def max_over_ranks(x: float, device=None) -> float:
    """The largest per-rank value over the process group (the job takes as long as its slowest rank);
    the value itself on a single process."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(n: int, n_bins: int, steps: int, world: int, seconds: float) -> float:
    """Whole-job neuron*bins/s: every rank processed steps x n x n_bins units in `seconds` (the max)."""
    return n * n_bins * steps * world / seconds


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, "fallback"


def cpu_model() -> str:
    """The host CPU's model name (lscpu; /proc/cpuinfo as a fallback)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_baseline(w, cores: int, n_rows: int | None = None, t_frac: float = 0.25):
    """The FP64 oracle as it stands, on a bounded sample: `cores` rows over the first t_frac of the bins."""
    import numpy as np
    import oracle
    n, T = w["n"], w["n_bins"]
    Ts = max(1, int(T * t_frac))
    offs, bins = w["offs"], w["bins"]
    # restrict the recording to its first Ts bins (a valid, shorter recording)
    keep = bins < Ts
    counts = np.array([keep[offs[i]:offs[i + 1]].sum() for i in range(n)], dtype=np.int64)
    offs_s = np.zeros(n + 1, dtype=np.int64)
    offs_s[1:] = np.cumsum(counts)
    bins_s = bins[keep]
    rows = np.linspace(0, n - 1, n_rows or cores).astype(np.int32)
    t0 = time.perf_counter()
    oracle.eval_rows(offs_s, bins_s, Ts, w["dt"], w["tau"], w["W_true"], w["b_true"], rows, threads=cores)
    el = time.perf_counter() - t0
    units = rows.size * Ts
    return {"value": units / el, "unit": UNIT, "cores": int(min(cores, rows.size)), "kind": "oracle",
            "sample": f"{rows.size} rows x first {Ts} of {T} bins (FP64 oracle, log-likelihood + gradient)",
            "seconds": el}


def cpu_baseline_report(w, cores: int, glm, device, stream, gpu_fit: dict | None, form: str = DEFAULT_FORM):
    """The CPU baseline of the bench line: the FP64 oracle timed on this host's cores, all cores and one
    thread, on bounded samples of the N = 1000 workload; the oracle's whole fit of the N = 50, 20 000-bin
    recording beside the GPU's fits of it (FP32 and the bench's form); and the N = 1000 evaluation and fit times
    extrapolated from the sampled rate (labelled as such: a full oracle evaluation takes minutes)."""
    import numpy as np
    import oracle
    import synth
    from synth import truth_labels
    allc = cpu_baseline(w, cores)
    one = cpu_baseline(w, 1, n_rows=1, t_frac=0.25)
    rep = {k: allc[k] for k in ("value", "unit", "cores", "kind", "sample")}
    rep["cpu_model"] = cpu_model()
    rep["single_thread"] = {"value": one["value"], "unit": UNIT, "cores": 1, "sample": one["sample"]}
    rep["all_core_over_single"] = allc["value"] / one["value"]
    # config 0: the whole fit, oracle (all cores and one thread) against the GPU
    w0 = synth.make_workload("glm_n50_t20k")
    truth0 = truth_labels(w0["W_true"])
    c0 = {"workload": "glm_n50_t20k (N = 50, 20 000 bins)", "eta": 1e-10}
    for label, th in (("oracle_all_cores", cores), ("oracle_one_thread", 1)):
        t0 = time.perf_counter()
        f = oracle.fit(w0["offs"], w0["bins"], w0["n_bins"], w0["dt"], w0["tau"], eta=1e-10, max_iter=500,
                       threads=th)
        el = time.perf_counter() - t0
        lab, _ = oracle.classify(f["W"], "gmm")
        c0[label] = {"seconds": el, "iterations_max": int(f["iters"].max()),
                     "mer": oracle.mer_breakdown(lab, truth0)["mer"]}
    oracle_labels = oracle.classify(f["W"], "gmm")[0]
    g = glm.GLM(device, stream=stream)
    try:
        for p in ("f32", form):
            g.set_problem(w0["offs"], w0["bins"], w0["n_bins"], w0["dt"], w0["tau"], prec=use_form(g, p))
            r = g.fit(eta=1e-10, max_iter=500)
            Wf = r["W"].cpu().numpy().astype(np.float64)
            lab, rr = glm.classify(Wf, "gmm", truth=truth0)
            c0[f"gpu_{p}"] = {"seconds": r["report"]["seconds"], "iterations": r["report"]["iterations"],
                              "mer": rr["mer"], "labels_equal_oracle": bool(np.array_equal(lab, oracle_labels))}
    finally:
        g.close()
    for p in ("f32", form):
        c0[f"oracle_all_cores_over_gpu_{p}"] = c0["oracle_all_cores"]["seconds"] / c0[f"gpu_{p}"]["seconds"]
    rep["config0_fit"] = c0
    # config 1 (N = 1000, 1.8 M bins): extrapolated from the sampled all-core rate
    s_eval = w["n"] * w["n_bins"] / allc["value"]
    ext = {"label": "extrapolated from the sampled all-core rate (not run)", "seconds_per_evaluation": s_eval}
    if gpu_fit and form in gpu_fit:
        ext[f"fit_seconds_at_gpu_{form}_evaluation_count"] = s_eval * gpu_fit[form]["evaluations"]
        ext[f"gpu_{form}_fit_seconds"] = gpu_fit[form]["seconds"]
    rep["config1_extrapolated"] = ext
    return rep


def run_reference(args):
    ws, rank, _ = dist_info()
    if rank != 0:
        return 0
    import synth
    w = synth.make_workload(args.workload)
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        cpu_baseline(w, cores, t_frac=0.05)
    vals, secs = [], 0.0
    for _ in range(args.steps):
        r = cpu_baseline(w, cores, t_frac=0.05)
        vals.append(r["value"])
        secs += r["seconds"]
    value = args.steps / sum(1.0 / v for v in vals)  # units per second over all steps
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "n": w["n"], "n_bins": w["n_bins"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": r["sample"], "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_batch(args, glm, device, form):
    """Uneven recordings (N ~ U{100..1500}, T ~ U(300, 3600) s x t_scale, 3-12 Hz) fitted one after another
    and then together with glm_fit_batch, to the same stopping rule; the speedup is the ratio of wall times."""
    import torch
    import synth
    specs = synth.batch_workloads(args.batch, t_scale=args.batch_t_scale)
    recs = [synth.make_workload(None, **sp) for sp in specs]
    ctxs = [glm.GLM(device) for _ in recs]
    try:
        for c, w in zip(ctxs, recs):
            c.set_problem(w["offs"], w["bins"], w["n_bins"], w["dt"], w["tau"], prec=use_form(c, form))
        kw = dict(eta=args.fit_eta, max_iter=args.fit_max_iter)
        torch.cuda.synchronize(device)
        t0 = time.perf_counter()
        seq = [c.fit(**kw)["report"] for c in ctxs]
        torch.cuda.synchronize(device)
        t_seq = time.perf_counter() - t0
        t0 = time.perf_counter()
        res, rc = glm.fit_batch(ctxs, **kw)
        torch.cuda.synchronize(device)
        t_bat = time.perf_counter() - t0
        # aggregate throughput of the fits: neuron-bins of every evaluation (trial points included) per second
        nb = [w["n"] * w["n_bins"] for w in recs]
        work_seq = sum(x * r["evaluations"] for x, r in zip(nb, seq))
        work_bat = sum(x * r["report"]["evaluations"] for x, r in zip(nb, res))
        return {"recordings": len(recs), "t_scale": args.batch_t_scale,
                "n": [w["n"] for w in recs], "n_bins": [w["n_bins"] for w in recs],
                "sequential_s": t_seq, "batched_s": t_bat, "speedup": t_seq / t_bat, "status": rc,
                "neuron_bins": sum(nb),
                "neuron_bins_per_s_sequential": work_seq / t_seq, "neuron_bins_per_s_batched": work_bat / t_bat,
                "evaluations_sequential": sum(r["evaluations"] for r in seq),
                "evaluations_batched": sum(r["report"]["evaluations"] for r in res),
                "iterations_max": max(r["report"]["iterations"] for r in res),
                "L_sequential": sum(r["L"] for r in seq), "L_batched": sum(r["report"]["L"] for r in res),
                "tile_choice": "autotuned inside glm_fit_batch (one row tile and units per SM for all problems)"}
    finally:
        for c in ctxs:
            c.close()


def run_ct(args, glm, w, device, stream, form):
    """The continuous-time form (event columns, exact interval integrals) on the first args.ct_seconds of the
    recording with its spikes moved off the grid, against the grid form on the same window: evaluation time,
    set-up time, U-product roofline, and a fit of each with its misclassification rate."""
    import numpy as np
    import torch
    import synth
    from synth import truth_labels
    n, dt, tau = w["n"], w["dt"], w["tau"]
    nb = min(w["n_bins"], int(round(args.ct_seconds / dt)))
    offs, bins = w["offs"], w["bins"]
    cnt = np.array([np.searchsorted(bins[offs[i]:offs[i + 1]], nb) for i in range(n)], dtype=np.int64)
    offs2 = np.zeros(n + 1, dtype=np.int64)
    offs2[1:] = np.cumsum(cnt)
    bins2 = np.concatenate([bins[offs[i]:offs[i] + cnt[i]] for i in range(n)]).astype(np.int32)
    times = synth.continuous_times(offs2, bins2, dt, 7)
    W = torch.from_numpy(w["W_true"].astype(np.float32)).cuda(device)
    b = torch.from_numpy(w["b_true"].astype(np.float32)).cuda(device)
    out = {"L_rows": torch.empty(n, dtype=torch.float64, device=device),
           "G": torch.empty((n, n), dtype=torch.float64, device=device),
           "gb": torch.empty(n, dtype=torch.float64, device=device)}
    res = {"workload": f"{args.workload}: first {nb * dt:g} s, spikes moved uniformly inside their bins, delay {dt:g} s",
           "spikes": int(offs2[-1])}
    k = max(3, args.steps)

    def timed(c):
        for _ in range(2):
            c.loglik_grad(W, b, total=False, out=out)
        torch.cuda.synchronize(device)
        c.profile(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            c.loglik_grad(W, b, total=False, out=out)
        e1.record(stream)
        torch.cuda.synchronize(device)
        prof = c.profile_read()
        c.profile(False)
        return e0.elapsed_time(e1) / k, {kk: v[1] / k for kk, v in prof.items()}

    truth = truth_labels(w["W_true"])
    ct = glm.GLM(device, stream=stream)
    gr = glm.GLM(device, stream=stream)
    try:
        torch.cuda.synchronize(device)
        t0 = time.perf_counter()
        ct.set_problem_ct(offs2, times, 0.0, nb * dt, tau, dt, prec=FORMS[form][0])  # columns always split
        torch.cuda.synchronize(device)
        res["setup_s"] = time.perf_counter() - t0
        M = ct.columns()
        ms, kern = timed(ct)
        peaks, src = measured_peaks()
        u_ms = kern.get("u_epilogue", float("nan"))
        ach = 6.0 * n * n * M / (u_ms / 1000.0) / 1e12
        res.update({"columns": M, "ms_per_eval": ms, "kernel_ms_per_eval": kern,
                    "neuron_columns_per_s": n * M / (ms / 1000.0),
                    "recording_seconds_per_s": nb * dt / (ms / 1000.0),
                    "u_product_roofline": {"bound": "tensor", "achieved": ach, "peak": peaks["bf16_tflops"],
                                           "unit": "TFLOP/s", "frac": ach / peaks["bf16_tflops"],
                                           "peak_source": f"{src} bf16_tflops (burst)"}})
        # one evaluation with dL/dtau as well (the U product's tau partials and their per-row scan)
        ct.loglik_grad(W, b, tau_grad=True)
        torch.cuda.synchronize(device)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            r_tau = ct.loglik_grad(W, b, tau_grad=True)
        e1.record(stream)
        torch.cuda.synchronize(device)
        res["with_dtau"] = {"ms_per_eval": e0.elapsed_time(e1) / k, "dL_dtau": r_tau["gtau"]}
        gr.set_problem(offs2, bins2, nb, dt, tau, prec=use_form(gr, form))
        gms, _ = timed(gr)
        res["grid_same_window"] = {"bins": nb, "ms_per_eval": gms}
        fits = {}
        Ws = {}
        for name, c in (() if args.no_ct_fit else (("continuous", ct), ("grid", gr))):
            r = c.fit(eta=args.fit_eta, max_iter=args.fit_max_iter)
            Wf = r["W"].cpu().numpy().astype(np.float64)
            _, rep = glm.classify(Wf, "gmm", truth=truth, types=w["types"])
            _, repk = glm.classify(Wf, "kmeans", truth=truth, types=w["types"])
            fits[name] = {"seconds": r["report"]["seconds"], "iterations": r["report"]["iterations"],
                          "evaluations": r["report"]["evaluations"], "mer_percent_gmm": 100.0 * rep["mer"],
                          "mer_percent_kmeans": 100.0 * repk["mer"], "centers_gmm": list(rep["centers"]),
                          "centers_kmeans": list(repk["centers"])}
            Ws[name] = r["W"]
        if Ws:
            dW = (Ws["continuous"] - Ws["grid"]).abs()
            fits["max_abs_W_difference"] = float(dW.max())
            fits["mean_abs_W_difference"] = float(dW.mean())
            res["fit"] = fits
    finally:
        ct.close()
        gr.close()
    return res


def run_classes(args, glm, w, device, stream, form, single_ms):
    """Per-neuron time constants and delays: the recording's rows split into args.classes classes of
    equal size, class k with tau = 8 + 2k ms and a delay of k + 1 bins, one context per class evaluating
    only its rows.  Times one evaluation of all classes (U products over each class's rows, E X^T over
    its row tiles, reductions) against the single-tau evaluation of the same recording."""
    import numpy as np
    import torch
    n, T = w["n"], w["n_bins"]
    K = args.classes
    cuts = [round(k * n / K) for k in range(K + 1)]
    W = torch.from_numpy(w["W_true"].astype(np.float32)).cuda(device)
    b = torch.from_numpy(w["b_true"].astype(np.float32)).cuda(device)
    outs = [{"L_rows": torch.empty(n, dtype=torch.float64, device=device),
             "G": torch.empty((n, n), dtype=torch.float64, device=device),
             "gb": torch.empty(n, dtype=torch.float64, device=device)} for _ in range(K)]
    ctxs = []
    try:
        torch.cuda.synchronize(device)
        t0 = time.perf_counter()
        for k in range(K):
            c = glm.GLM(device, stream=stream)
            ctxs.append(c)
            c.set_source_delay(k + 1)
            c.set_problem(w["offs"], w["bins"], T, w["dt"], 0.008 + 0.002 * k, prec=use_form(c, form))
            c.set_row_range(cuts[k], cuts[k + 1])
        torch.cuda.synchronize(device)
        setup_s = time.perf_counter() - t0
        for _ in range(2):
            for c, o in zip(ctxs, outs):
                c.loglik_grad(W, b, total=False, out=o)
        steps = max(3, args.steps)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(device)
        e0.record(stream)
        for _ in range(steps):
            for c, o in zip(ctxs, outs):
                c.loglik_grad(W, b, total=False, out=o)
        e1.record(stream)
        torch.cuda.synchronize(device)
        ms = e0.elapsed_time(e1) / steps
    finally:
        for c in ctxs:
            c.close()
    return {"classes": K, "rows": [cuts[k + 1] - cuts[k] for k in range(K)],
            "tau_ms": [8 + 2 * k for k in range(K)], "delay_bins": [k + 1 for k in range(K)],
            "setup_s": setup_s, "ms_per_eval_all_classes": ms, "single_tau_ms_per_eval": single_ms,
            "neuron_bins_per_s": n * T / (ms / 1000.0)}


def run_undersampling(args, glm, w, device, stream, form):
    """Undersampling (App. C.2): fit only the spike trains of a random subset of the neurons (excitatory
    and inhibitory in their full proportion), classify the subset's weights against the generating ones."""
    import numpy as np
    from synth import truth_labels
    rng = np.random.default_rng(17)
    exc = np.nonzero(w["types"] > 0)[0]
    inh = np.nonzero(w["types"] < 0)[0]
    out = []
    for f in [float(x) for x in args.undersampling.split(",") if x]:
        sub = np.sort(np.concatenate([rng.choice(exc, int(round(f * len(exc))), replace=False),
                                      rng.choice(inh, int(round(f * len(inh))), replace=False)]))
        offs = np.zeros(len(sub) + 1, dtype=np.int64)
        offs[1:] = np.cumsum([w["offs"][i + 1] - w["offs"][i] for i in sub])
        bins = np.concatenate([w["bins"][w["offs"][i]:w["offs"][i + 1]] for i in sub]).astype(np.int32)
        c = glm.GLM(device, stream=stream)
        try:
            c.set_problem(offs, bins, w["n_bins"], w["dt"], w["tau"], prec=use_form(c, form))
            r = c.fit(eta=args.fit_eta, max_iter=args.fit_max_iter)
        finally:
            c.close()
        Wf = r["W"].cpu().numpy().astype(np.float64)
        truth = truth_labels(w["W_true"][np.ix_(sub, sub)])
        _, rg = glm.classify(Wf, "gmm", truth=truth, types=w["types"][sub])
        _, rk = glm.classify(Wf, "kmeans", truth=truth, types=w["types"][sub])
        out.append({"fraction": f, "neurons": int(len(sub)), "fit_seconds": r["report"]["seconds"],
                    "mer_gmm": rg["mer"], "mer_kmeans": rk["mer"]})
    return out


def chain_links(W_true, w_syn):
    """The links of the planted synfire chain, in chain order, from the generating weights: every neuron of
    link g + 1 receives exactly w_syn from every neuron of link g (no other weight has that value)."""
    import numpy as np
    hit = np.isclose(W_true, w_syn)
    targets = {}
    for j in np.nonzero(hit.any(axis=0))[0]:
        targets.setdefault(tuple(np.nonzero(hit[:, j])[0]), []).append(int(j))
    groups = {frozenset(v): frozenset(k) for k, v in targets.items()}  # link -> next link
    heads = [g for g in groups if not any(g <= nxt for nxt in groups.values())]
    links = [heads[0]] if heads else []
    while links and links[-1] in groups:
        links.append(groups[links[-1]])
    return [sorted(l) for l in links]


def links_found(Z, links, m):
    """Links that some subtree of the dendrogram holds >= 90 % of while being >= 90 % pure."""
    work = {k: {k} for k in range(m)}
    subtrees = []
    for q, (a, b, _, _) in enumerate(Z):
        c = work.pop(int(a)) | work.pop(int(b))
        work[m + q] = c
        if len(c) <= 4 * max(len(l) for l in links):
            subtrees.append(c)
    found = []
    for l in links:
        L = set(l)
        ok = any(len(c & L) >= 0.9 * len(L) and len(c & L) >= 0.9 * len(c) for c in subtrees)
        found.append(bool(ok))
    return found


def run_synfire(args, glm, device, stream, form):
    """The synfire recording (N = 2000 with a 10 x 50 chain, ids shuffled, as in Sec. 3.4): fit, classify,
    and find the chain's links by Ward clustering of the fitted weights, by outgoing connections (links
    that project to a next link) and by incoming ones (links that receive from a previous link)."""
    import numpy as np
    import torch
    import synth
    from synth import truth_labels
    cfg = synth.WORKLOADS["glm_n2000_synfire_t3600s"]
    nb = int(round(args.synfire_seconds / cfg["dt"]))
    t0 = time.perf_counter()
    w = synth.make_workload("glm_n2000_synfire_t3600s", n_bins=nb)
    gen_s = time.perf_counter() - t0
    links = chain_links(w["W_true"], cfg["w_syn"])
    c = glm.GLM(device, stream=stream)
    try:
        c.set_problem(w["offs"], w["bins"], nb, w["dt"], w["tau"], prec=use_form(c, form))
        r = c.fit(eta=args.fit_eta, max_iter=args.fit_max_iter)
        Wf = r["W"]
        Wn = Wf.cpu().numpy().astype(np.float64)
        truth = truth_labels(w["W_true"])
        _, rep = glm.classify(Wn, "gmm", truth=truth, types=w["types"])
        _, rep_k = glm.classify(Wn, "kmeans", truth=truth, types=w["types"])
        torch.cuda.synchronize(device)
        t1 = time.perf_counter()
        Zo = c.ward(Wf, by="out")
        Zi = c.ward(Wf, by="in")
        ward_s = time.perf_counter() - t1
    finally:
        c.close()
    fo, fi = links_found(Zo, links, w["n"]), links_found(Zi, links, w["n"])
    return {"workload": f"glm_n2000_synfire: N = 2000, {nb * cfg['dt']:g} s, 10 x 50 synfire links, ids shuffled",
            "generation_s": gen_s, "fit": {"seconds": r["report"]["seconds"], "iterations": r["report"]["iterations"],
                                           "evaluations": r["report"]["evaluations"], "mer": rep["mer"],
                                           "mer_kmeans": rep_k["mer"], "converged": r["report"]["converged"],
                                           "at_floor": r["report"]["at_floor"], "maxiter": r["report"]["maxiter"],
                                           "centers_gmm": list(rep["centers"])},
            "ward_seconds_two_linkages": ward_s,
            "links": len(links), "found_by_outgoing": fo, "found_by_incoming": fi,
            "found_by_either": int(sum(a or b for a, b in zip(fo, fi)))}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import numpy as np
    import torch
    import torch.distributed as dist

    import synth
    import paper_1502_04993_gb300 as glm

    ws, rank, local = dist_info()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    device = local if ws > 1 else 0
    torch.cuda.set_device(device)
    form = args.prec or DEFAULT_FORM
    prec, xsplit = FORMS[form]
    cfg = dict(synth.WORKLOADS[args.workload])
    extra = {"n_bins": args.n_bins} if args.n_bins else {}
    w = synth.make_workload(args.workload, seed=rank_seed(cfg["seed"], rank), **extra)  # independent recording per rank
    n, T = w["n"], w["n_bins"]
    stream = torch.cuda.current_stream(device)
    ctx = glm.GLM(device, stream=stream)
    use_form(ctx, form)
    ctx.set_problem(w["offs"], w["bins"], T, w["dt"], w["tau"], prec=prec)
    W = torch.from_numpy(w["W_true"].astype(np.float32)).cuda(device)
    b = torch.from_numpy(w["b_true"].astype(np.float32)).cuda(device)
    out = {"L_rows": torch.empty(n, dtype=torch.float64, device=device),
           "G": torch.empty((n, n), dtype=torch.float64, device=device),
           "gb": torch.empty(n, dtype=torch.float64, device=device)}

    def step():
        ctx.prepare()
        ctx.loglik_grad(W, b, total=False, out=out)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize(device)
    if ws > 1:
        dist.barrier()
    clocks = Clocks(device)
    clocks.start()
    ctx.profile(True)
    launches0 = ctx.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(device)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize(device)
    ms = ev0.elapsed_time(ev1)
    launches = ctx.launch_count() - launches0
    prof = ctx.profile_read()
    ctx.profile(False)
    clk = clocks.stop()
    ms = max_over_ranks(ms, device)
    if ws > 1:
        dist.barrier()
    value = job_throughput(n, T, args.steps, ws, ms / 1000.0)

    # ---- the evaluation alone, X already filtered (what every fit iteration repeats) ----
    torch.cuda.synchronize(device)
    ev2, ev3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev2.record(stream)
    for _ in range(args.steps):
        ctx.loglik_grad(W, b, total=False, out=out)
    ev3.record(stream)
    torch.cuda.synchronize(device)
    ms_eval = max_over_ranks(ev2.elapsed_time(ev3), device)

    # ---- end to end through the public API from host buffers ----
    k2 = args.e2e_steps or max(1, min(args.steps, 5))
    W_h = torch.from_numpy(w["W_true"].astype(np.float32)).pin_memory()
    b_h = torch.from_numpy(w["b_true"].astype(np.float32)).pin_memory()
    G_h = torch.empty((n, n), dtype=torch.float64).pin_memory()
    offs_h = torch.from_numpy(w["offs"]).pin_memory().numpy()  # the step's inputs in pinned host memory
    bins_h = torch.from_numpy(w["bins"]).pin_memory().numpy()
    torch.cuda.synchronize(device)
    if ws > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(k2):
        ctx.set_problem(offs_h, bins_h, T, w["dt"], w["tau"], prec=prec)
        Wd = W_h.to(device, non_blocking=True)
        bd = b_h.to(device, non_blocking=True)
        r = ctx.loglik_grad(Wd, bd, total=True, out=out)
        G_h.copy_(r["G"], non_blocking=True)
        torch.cuda.synchronize(device)
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, device)
    h2d = w["offs"].nbytes + w["bins"].nbytes + W_h.numel() * 4 + b_h.numel() * 4
    d2h = G_h.numel() * 8 + 8

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return 0

    # ---- roofline of the dominant kernel group ----
    peaks, peak_src = measured_peaks()
    top = max(prof.items(), key=lambda kv: kv[1][1])
    name, (cnt, tot_ms) = top
    per_launch_s = tot_ms / cnt / 1000.0
    if name in ("u_epilogue", "grad"):
        if prec == "f32":
            flops = 2.0 * n * n * T
            # FP32 FMA pipes: 152 SMs x 128 lanes x 2 flop x max SM clock
            sm_mhz = peaks.get("sm_max_mhz", 2070.0)
            peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
            roof = {"bound": "alu", "achieved": flops / per_launch_s / 1e12, "peak": peak, "unit": "TFLOP/s",
                    "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x max SM clock"}
        else:
            # algorithmic work per neuron-bin: 2N for the plain product; the U product with W as hi + lo
            # (W_hi X + W_lo X) is 4N.  With X split the kernel also executes W_hi X_lo (the rounding
            # correction of X): 6N executed.
            alg = 4.0 if name == "u_epilogue" else 2.0
            executed = (6.0 if xsplit else 4.0) if name == "u_epilogue" else 2.0
            peak = peaks["bf16_tflops"]
            ach = alg * n * n * T / per_launch_s / 1e12
            roof = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                    "peak_source": f"{peak_src} bf16_tflops (burst)",
                    "flop_count": (f"{alg:g}N per neuron-bin (W_hi X + W_lo X)" if name == "u_epilogue"
                                   else "2N per neuron-bin")}
            ex = executed * n * n * T / per_launch_s / 1e12
            roof["executed"] = {"achieved": ex, "frac": ex / peak,
                                "flop_count": f"{executed:g}N per neuron-bin, every product the kernel issues"}
            if name == "u_epilogue":
                roof["plain_2N_frac"] = 2.0 * n * n * T / per_launch_s / 1e12 / peak
            pk = peaks.get("clocks_under_load", {}).get("sm_mhz_median")
            if pk and clk.get("sm_mhz"):
                # the peak was measured at its own clock: scaled to this run's median SM clock
                roof["clock_normalised"] = {"peak_run_sm_mhz": pk, "this_run_sm_mhz": clk["sm_mhz"],
                                            "frac": ach / (peak * clk["sm_mhz"] / pk)}
    else:
        esz = 4 if prec == "f32" else 2
        # the filter writes X once in its stored type (the algorithmic bytes) and reads the spikes
        nbytes = {"filter_scan": n * T * esz + w["bins"].nbytes,
                  "spike_term": w["bins"].nbytes * (n // 8 + 1)}.get(name, n * T * esz)
        peak = peaks["hbm_gbs"]
        roof = {"bound": "hbm", "achieved": nbytes / per_launch_s / 1e9, "peak": peak, "unit": "GB/s",
                "peak_source": f"{peak_src} hbm_gbs"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    # DRAM bytes per launch of the dominant kernel from one ncu capture (dram__bytes_read.sum +
    # dram__bytes_write.sum), N = 1000 x 200 000 bins, scaled to the launch by its neuron-bins (the traffic
    # of these kernels grows in proportion: X read once, the rates written once); None for kernels not
    # captured in their present form
    traffic_per_unit = {("u_epilogue", "f16x1"): (415.170048e6 + 363.148544e6) / (1000 * 200000)}
    tpu = traffic_per_unit.get((name, form))
    roof["traffic"] = tpu * n * T if tpu is not None else None
    roof["kernel"] = name
    roof["ms_per_launch"] = tot_ms / cnt

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": prec, "data": "synthetic",
        "config": {"workload": args.workload, "n": n, "n_bins": T, "precision": prec, "form": form,
                   "x_storage": ("FP32 X" if prec == "f32" else
                                 f"X as {prec} X_hi + X_lo" if xsplit else f"X as one {prec} array"),
                   "l2": "inputs larger than L2 (filtered trains %.1f GB)" % (n * T * (2 if prec != "f32" and not xsplit else 4) / 1e9),
                   "parallelism": f"replicas x{ws}: one independent recording per GPU"},
        "e2e": {"value": job_throughput(n, T, k2, ws, e2e_s), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "steps": k2},
        "gpu_launches": int(launches),
        "x_cached": {"value": job_throughput(n, T, args.steps, ws, ms_eval / 1000.0), "unit": UNIT,
                     "ms_per_eval": ms_eval / args.steps,
                     "what": "glm_loglik_grad with gradient on the filtered X already in HBM (one fit evaluation)"},
        "kernel_ms_per_step": {k: v[1] / args.steps for k, v in prof.items()},
        "roofline": roof,
        "clocks": clk,
    }
    if args.fit:
        # full fits: wall time of glm_fit per precision, and the classification against the ground truth
        from synth import truth_labels
        truth = truth_labels(w["W_true"])
        fits = {}
        fit_params = {}
        for p in [s for s in args.fit.split(",") if s]:
            ctx.set_problem(w["offs"], w["bins"], T, w["dt"], w["tau"], prec=use_form(ctx, p))
            torch.cuda.synchronize(device)
            r = ctx.fit(eta=args.fit_eta, max_iter=args.fit_max_iter)
            fit_params[p] = (r["W"], r["b"])
            Wf = r["W"].cpu().numpy().astype(np.float64)
            _, rep = glm.classify(Wf, "gmm", truth=truth, types=w["types"])
            fr = r["report"]
            fits[p] = {"seconds": fr["seconds"], "iterations": fr["iterations"], "evaluations": fr["evaluations"],
                       "gradients": fr["gradients"], "converged": fr["converged"], "at_floor": fr["at_floor"], "stalled": fr["stalled"],
                       "maxiter": fr["maxiter"], "L": fr["L"], "mer": rep["mer"], "mer_percent": 100.0 * rep["mer"],
                       "mer_n2": rep["mer_n2"]}
        base = next((p for p in fits if p != "f32"), None)
        if "f32" in fits and base is not None:
            # the 16-bit fit finished by the plain FP32 form from its result (warm start): the 16-bit
            # objective's optimum lies a few 1e-7 of L below the exact one; FP32 iterations close that gap
            torch.cuda.synchronize(device)
            t0 = time.perf_counter()
            ctx.set_problem(w["offs"], w["bins"], T, w["dt"], w["tau"], prec=use_form(ctx, "f32"))
            rp = ctx.fit(fit_params[base][0], fit_params[base][1], eta=args.fit_eta, max_iter=args.fit_max_iter)
            torch.cuda.synchronize(device)
            t_polish = time.perf_counter() - t0
            Wf = rp["W"].cpu().numpy().astype(np.float64)
            _, rep = glm.classify(Wf, "gmm", truth=truth, types=w["types"])
            fr = rp["report"]
            fits[f"{base}+f32_polish"] = {"seconds": fits[base]["seconds"] + t_polish, "polish_seconds": t_polish,
                                          "polish_iterations": fr["iterations"], "evaluations": fr["evaluations"],
                                          "converged": fr["converged"], "at_floor": fr["at_floor"],
                                          "mer": rep["mer"], "mer_percent": 100.0 * rep["mer"]}
            fit_params[f"{base}+f32_polish"] = (rp["W"], rp["b"])
        if "f32" in fits:
            for p, v in fits.items():
                v["speedup_vs_f32"] = fits["f32"]["seconds"] / v["seconds"]
            # every fit's W, b scored by one evaluation, the plain FP32 form's (L within ~1e-9 of exact): the
            # fits' own final L each carry their form's evaluation error and are not comparable at 1e-8
            ctx.set_problem(w["offs"], w["bins"], T, w["dt"], w["tau"], prec=use_form(ctx, "f32"))
            for p, (Wf, bf) in fit_params.items():
                rr = ctx.loglik_grad(Wf, bf, grad=False)
                fits[p]["L_scored_f32"] = rr["L_total"]
            for p in fits:
                fits[p]["L_gap_to_f32_fit"] = (fits["f32"]["L_scored_f32"] - fits[p]["L_scored_f32"]) / abs(fits["f32"]["L_scored_f32"])
        line["fit"] = {"eta": args.fit_eta, "max_iter": args.fit_max_iter, "by_precision": fits}
    if args.batch:
        line["batch"] = run_batch(args, glm, device, form)
    if args.ct_seconds > 0 and prec != "f32":
        line["continuous_time"] = run_ct(args, glm, w, device, stream, form)
    if args.classes > 0 and prec != "f32":
        line["row_classes"] = run_classes(args, glm, w, device, stream, form, ms_eval / args.steps)
    if args.undersampling:
        line["undersampling"] = run_undersampling(args, glm, w, device, stream, form)
    if args.synfire:
        line["synfire"] = run_synfire(args, glm, device, stream, form)
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_report(w, os.cpu_count() or 1, glm, device, stream,
                                                   line.get("fit", {}).get("by_precision"),
                                                   form if prec != "f32" else DEFAULT_FORM)
    print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
