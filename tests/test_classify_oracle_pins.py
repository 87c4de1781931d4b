"""Pins of the oracle's 1-D classifiers (Sec. 3.1 Gaussian mixture by EM, Sec. 3.3 / App. C.2 k-means with
k = 3) to facts fixed outside them: recovery of a known mixture within its sampling error, the EM fixed
point and the monotone log-likelihood that define EM, a Lloyd run worked out by hand (percentile start and
the tie rule that sends an equidistant point to the centre nearer zero), and exact posterior ties.  The
densities here come from scipy.stats, not from the oracle's formula.  The library's classifier (host code
in libglm) must give the same labels on the hand-worked and tie cases."""
import math

import numpy as np
import pytest
from scipy import stats
from scipy.special import logsumexp

import oracle
from oracle.classify import gmm_assign, gmm1d, kmeans1d

# a known 3-component mixture, ordered by mean (inhibitory, absent, excitatory)
PI = np.array([0.10, 0.75, 0.15])
MU = np.array([-0.8, 0.0, 0.2])
SD = np.array([0.05, 0.03, 0.04])
N_DRAWS = 200_000


@pytest.fixture(scope="module")
def mixture_sample():
    rng = np.random.default_rng(2024)
    k = rng.choice(3, size=N_DRAWS, p=PI)
    return rng.normal(MU[k], SD[k])


@pytest.fixture(scope="module")
def mixture_fit(mixture_sample):
    trace = []
    (pi, mu, var), assign, ll = gmm1d(mixture_sample, trace=trace)
    return dict(pi=pi, mu=mu, var=var, assign=assign, ll=ll, trace=trace)


def test_gmm_recovers_known_mixture_within_sampling_error(mixture_fit):
    """Each parameter within 5 standard errors of the generating value: SE(pi_k) = sqrt(pi(1-pi)/n),
    SE(mu_k) = sd_k / sqrt(n pi_k), SE(var_k) = var_k sqrt(2 / (n pi_k)).  A wrong M step (a weight not
    normalised by n, a variance not centred or not divided by the component's mass, a dropped 1/2 in
    the exponent) misses these by far more."""
    n = N_DRAWS
    f = mixture_fit
    se_pi = np.sqrt(PI * (1 - PI) / n)
    se_mu = SD / np.sqrt(n * PI)
    se_var = SD ** 2 * np.sqrt(2.0 / (n * PI))
    assert np.all(np.abs(f["pi"] - PI) < 5 * se_pi), (f["pi"], PI)
    assert np.all(np.abs(f["mu"] - MU) < 5 * se_mu), (f["mu"], MU)
    assert np.all(np.abs(f["var"] - SD ** 2) < 5 * se_var), (f["var"], SD ** 2)
    assert f["pi"].sum() == pytest.approx(1.0, abs=1e-12)


def test_gmm_converges_to_an_em_fixed_point(mixture_sample, mixture_fit):
    """At convergence the parameters reproduce themselves: responsibilities computed from them (scipy's
    normal density) give back the same weights, means and variances."""
    x = mixture_sample
    f = mixture_fit
    logp = np.log(f["pi"])[None, :] + stats.norm.logpdf(x[:, None], f["mu"][None, :], np.sqrt(f["var"])[None, :])
    r = np.exp(logp - logsumexp(logp, axis=1, keepdims=True))
    nk = r.sum(axis=0)
    pi2 = nk / x.size
    mu2 = (r * x[:, None]).sum(axis=0) / nk
    var2 = (r * (x[:, None] - mu2[None, :]) ** 2).sum(axis=0) / nk
    assert np.allclose(pi2, f["pi"], rtol=1e-6, atol=0)
    assert np.allclose(mu2, f["mu"], rtol=0, atol=1e-6 * SD.min())
    assert np.allclose(var2, f["var"], rtol=1e-5, atol=0)


def test_gmm_log_likelihood_never_decreases(mixture_sample, mixture_fit):
    """EM's defining property: the mixture log-likelihood of successive iterates is non-decreasing, and the
    returned parameters are at least as likely as the last iterate (scipy's density)."""
    tr = np.array(mixture_fit["trace"])
    assert tr.size >= 2
    assert np.all(np.diff(tr) >= -1e-12 * np.abs(tr[1:])), np.diff(tr).min()
    f = mixture_fit
    logp = np.log(f["pi"])[None, :] + stats.norm.logpdf(mixture_sample[:, None], f["mu"][None, :],
                                                         np.sqrt(f["var"])[None, :])
    ll_final = logsumexp(logp, axis=1).sum()
    assert ll_final >= tr[-1] - 1e-12 * abs(tr[-1])
    assert ll_final == pytest.approx(f["ll"], rel=1e-9)


def test_gmm_labels_match_bayes_rule_of_the_true_mixture(mixture_sample, mixture_fit):
    """With ~1e5 draws the fitted mixture's decisions equal those of the generating mixture except for
    points in the thin band where the two posteriors cross."""
    x = mixture_sample
    logp = np.log(PI)[None, :] + stats.norm.logpdf(x[:, None], MU[None, :], SD[None, :])
    bayes = logp.argmax(axis=1)
    assert np.mean(bayes != mixture_fit["assign"]) < 1e-3


KMEANS_HAND_CASES = [
    # x, initial centroids (1st, 50th, 99th percentiles, linear interpolation), final centroids, final clusters.
    # 0..10: start (0.1, 5, 9.9) -> {0,1,2} {3..7} {8,9,10} -> means (1, 5, 9); 3 and 7 are then equidistant
    # from two centres and join the one nearer zero -> {0..3} {4..7} {8..10} -> (1.5, 5.5, 9), stable.
    (np.arange(11.0), (0.1, 5.0, 9.9), (1.5, 5.5, 9.0), [0] * 4 + [1] * 4 + [2] * 3),
    # -10..0: the mirror image.  The ties (-7 between -9 and -5, -3 between -5 and -1) again join the centre
    # nearer zero, which here is the later one: (-9, -5.5, -1.5).  Taking the first of two equal distances
    # instead would end at (-8.5, -4.5, -1).
    (np.arange(-10.0, 1.0), (-9.9, -5.0, -0.1), (-9.0, -5.5, -1.5), [0] * 3 + [1] * 4 + [2] * 4),
]


@pytest.mark.parametrize("x,c0,cfin,clusters", KMEANS_HAND_CASES)
def test_kmeans_hand_worked_lloyd_run(x, c0, cfin, clusters):
    c_init, _ = kmeans1d(x, max_iter=0)
    assert np.allclose(c_init, c0, rtol=0, atol=1e-12)
    c, assign = kmeans1d(x)
    assert np.allclose(c, cfin, rtol=0, atol=1e-12)
    assert assign.tolist() == clusters


def test_gmm_posterior_tie_goes_to_component_nearer_zero():
    """Equal weights and variances, means -1, 0, 1: -0.5 and 0.5 have exactly equal posteriors under two
    components and are assigned to the middle one (mean 0, 'absent'); -2 and 2 go to the outer ones."""
    pi = np.full(3, 1.0 / 3.0)
    mu = np.array([-1.0, 0.0, 1.0])
    var = np.ones(3)
    assert gmm_assign(np.array([-0.5, 0.5, -2.0, 2.0, 0.0]), pi, mu, var).tolist() == [1, 1, 0, 2, 1]


@pytest.fixture(scope="module")
def glm():
    from paper_1502_04993_gb300 import build as b
    import paper_1502_04993_gb300 as g
    g.load_library(b.build())
    return g


@pytest.mark.parametrize("case", range(len(KMEANS_HAND_CASES)))
def test_library_kmeans_on_hand_worked_runs(glm, case):
    """The library's 3-means labels the hand-worked data as the worked run does, ties included (the values
    sit off the diagonal of a 4 x 4 matrix, with one more copy of the final middle centre as the twelfth),
    and agrees with the oracle's centres."""
    x, _, cfin, clusters = KMEANS_HAND_CASES[case]
    n = 4  # 12 off-diagonal entries: the 11 values plus one more copy of the middle centre
    vals = np.concatenate([x, [cfin[1]]])
    W = np.zeros((n, n))
    W[~np.eye(n, dtype=bool)] = vals
    lab, rep = glm.classify(W, "kmeans")
    lab_o, model = oracle.classify(W, "kmeans")
    assert np.array_equal(lab, lab_o)
    assert np.allclose(rep["centers"], model["centroids"], rtol=0, atol=1e-12)
    got = lab[~np.eye(n, dtype=bool)][:11] + 1
    assert got.tolist() == clusters
