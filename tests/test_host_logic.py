"""Host-side logic that needs no GPU: splitting a recording for cross-validation, the generator's ground-truth
labels, and the double-float arithmetic of the segment carries."""
import numpy as np
import pytest

import synth


def test_split_recording_conserves_and_rebases():
    import paper_1502_04993_gb300 as glm
    w = synth.make_workload("glm_n50_t20k")
    (a, b) = glm.split_recording(w["offs"], w["bins"], w["n_bins"], 12000)
    assert a[2] == 12000 and b[2] == w["n_bins"] - 12000
    assert a[0][-1] + b[0][-1] == w["offs"][-1]
    n = w["offs"].size - 1
    for i in range(n):
        row = w["bins"][w["offs"][i]:w["offs"][i + 1]]
        ra = a[1][a[0][i]:a[0][i + 1]]
        rb = b[1][b[0][i]:b[0][i + 1]]
        assert np.array_equal(np.concatenate([ra, rb + 12000]), row)
        assert np.all(ra < 12000) and np.all(rb >= 0) and np.all(rb < b[2])


def test_split_recording_ct():
    import paper_1502_04993_gb300 as glm
    offs = np.array([0, 3, 3, 5], dtype=np.int64)
    times = np.array([0.1, 0.5, 0.9, 0.45, 0.7])
    (o1, t1, a1, b1), (o2, t2, a2, b2) = glm.split_recording_ct(offs, times, 0.0, 1.0, 0.5)
    assert o1.tolist() == [0, 1, 1, 2] and t1.tolist() == [0.1, 0.45] and (a1, b1) == (0.0, 0.5)
    assert o2.tolist() == [0, 2, 2, 3] and t2.tolist() == [0.5, 0.9, 0.7] and (a2, b2) == (0.5, 1.0)


def test_synth_truth_labels_match_the_oracle_definition():
    """The bench's ground-truth labels (from the generator) agree with the oracle's classification truth."""
    import synth
    from oracle.classify import truth_labels
    rng = np.random.default_rng(0)
    W = rng.choice([-1.2, 0.0, 0.3], size=(37, 37), p=[0.1, 0.8, 0.1])
    np.fill_diagonal(W, -3.0)
    assert np.array_equal(synth.truth_labels(W), truth_labels(W))


def _df_add(a, b):
    """Double-float sum of FP32 pairs, the steps of df_add in the CUDA scan header (TwoSum, then a renormalising
    fast two-sum), evaluated in numpy float32."""
    f = np.float32
    s = f(a[0] + b[0])
    bp = f(s - a[0])
    e = f(f(a[0] - f(s - bp)) + f(b[0] - bp))
    e = f(e + f(a[1] + b[1]))
    h = f(s + e)
    return (h, f(e - f(h - s)))


def _df_mul(a, b):
    """Double-float product (Dekker): the exact error of the FP32 product by an FMA, evaluated exactly in FP64
    and rounded once, as fmaf does."""
    f = np.float32
    p = f(a[0] * b[0])
    e = f(float(a[0]) * float(b[0]) - float(p))          # fmaf(a.x, b.x, -p): exact product minus p, rounded
    e = f(float(a[1]) * float(b[0]) + float(e))          # fmaf(a.y, b.x, e)
    e = f(float(a[0]) * float(b[1]) + float(e))          # fmaf(a.x, b.y, ...)
    h = f(p + e)
    return (h, f(e - f(h - p)))


def _df(v):
    h = np.float32(v)
    return (h, np.float32(v - float(h)))


@pytest.mark.parametrize("tau_over_dt", [10.0, 1000.0, 100000.0])
def test_double_float_segment_carries_track_fp64(tau_over_dt):
    """The segment carries X[256 (s+1)] = A X[256 s] + local[s] run in double-float pairs on the device; over a
    few thousand segments, even with A close to 1 (tau of 10^5 bins, where errors accumulate), the pair stays
    within a small multiple of 2^-44 of the FP64 recursion (relative, for values in FP32's normal range), far
    below the FP32 rounding its readers apply."""
    rng = np.random.default_rng(1)
    a_seg = np.exp(-256.0 / tau_over_dt)
    A = _df(a_seg)
    x64, x = 0.0, (np.float32(0), np.float32(0))
    worst = 0.0
    for s in range(3000):
        loc = float(rng.exponential(1.0)) * float(rng.random() < 0.9)
        x64 = a_seg * x64 + loc
        x = _df_add(_df_mul(A, x), _df(loc))
        # relative to the value, above FP32's normal range (a run of empty segments with a tiny A takes the pair
        # into FP32's subnormals, where it keeps an absolute accuracy of ~1e-45 that no reader can see)
        worst = max(worst, abs((float(x[0]) + float(x[1])) - x64) / (x64 + 2.0 ** -100))
    assert worst < 2.0 ** -40, worst


def test_fp32_form_expm1_is_correctly_rounded():
    """The plain FP32 form's e^v - 1 (glm_expm1, the epilogue's own source run on the host) against e^v - 1 in
    FP64 rounded once to FP32: equal but for rare near-ties (never more than one ulp away), and unbiased (mean
    signed error ~0 ulp; CUDA's expm1f measured -0.035 ulp on this range, enough to bias L by ~5e-10)."""
    import numpy as np
    from paper_1502_04993_gb300 import build as b
    import paper_1502_04993_gb300 as glm
    glm.load_library(b.build())
    rng = np.random.default_rng(5)
    v = np.concatenate([np.linspace(-0.6, 1.5, 400_001), rng.uniform(-19.9, 88.0, 200_000),
                        rng.normal(0, 1e-3, 50_000), [0.0, -0.0, 1e-30, -1e-30, 0.34657, -0.34658, 88.0, -20.0]])
    v = v.astype(np.float32)
    got = glm.expm1(v).astype(np.float64)
    ref32 = np.expm1(v.astype(np.float64)).astype(np.float32).astype(np.float64)
    ulp = np.spacing(np.abs(ref32).astype(np.float32)).astype(np.float64)
    ex = np.expm1(v.astype(np.float64))
    d = (got - ex) / ulp
    assert np.mean(got != ref32) < 1e-3
    assert np.max(np.abs(got - ref32) / ulp) <= 1.0
    assert abs(np.mean(d)) < 2e-3
    assert glm.expm1(np.array([np.nan, 100.0, -50.0], np.float32)).tolist()[1:] == [np.inf, -1.0]
