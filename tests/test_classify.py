"""glm_classify (host code in libglm) against the oracle's classifier on the same weights: identical labels
and cluster centres, and the same error breakdown.  Runs without a GPU."""
import numpy as np
import pytest

import oracle
import synth
from oracle.classify import truth_labels


@pytest.fixture(scope="module")
def glm():
    from paper_1502_04993_gb300 import build as b
    import paper_1502_04993_gb300 as g
    g.load_library(b.build())
    return g


def noisy_weights(n, seed, sd):
    W, types = synth.network(n, int(0.8 * n), 0.1, 0.2, 0.8, seed=seed)
    rng = np.random.default_rng(seed)
    return W + rng.normal(0, sd, W.shape), W, types


@pytest.mark.parametrize("method", ["gmm", "kmeans"])
@pytest.mark.parametrize("n,seed,sd", [(60, 1, 0.03), (200, 2, 0.06), (300, 3, 0.1)])
def test_classify_matches_oracle(glm, method, n, seed, sd):
    Wn, Wt, types = noisy_weights(n, seed, sd)
    truth = truth_labels(Wt)
    lab, rep = glm.classify(Wn, method, truth=truth, types=types)
    lab_o, model = oracle.classify(Wn, method)
    assert np.array_equal(lab, lab_o)
    centers_o = model["centroids"] if method == "kmeans" else model["means"]
    assert np.allclose(rep["centers"], centers_o, rtol=1e-9, atol=1e-12)
    br = oracle.mer_breakdown(lab_o, truth, types)
    assert rep["errors"] == br["errors"] and rep["mer"] == pytest.approx(br["mer"])
    assert rep["mer_n2"] == pytest.approx(br["mer_n2"])
    for nm in ("exc", "inh", "absent"):
        assert (rep[nm]["fp"], rep[nm]["fn"]) == (br[nm]["fp"], br[nm]["fn"])
    for nm in ("exc", "inh"):
        assert rep[nm]["nd"] == br[nm]["nd"]


def test_classify_errors(glm):
    with pytest.raises(glm.GLMError):
        glm.classify(np.zeros((1, 1)))
    W = np.zeros((3, 3))
    W[0, 1] = np.nan
    with pytest.raises(glm.GLMError) as e:
        glm.classify(W)
    assert e.value.code == -6
