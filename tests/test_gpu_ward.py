"""Ward clustering of neurons by their weights on the GPU (glm_ward, glm_ward_cut) against the FP64 oracle
(oracle.ward, itself pinned to SciPy's linkage), and the synfire-chain identification it serves (Sec.
3.4.2): in a network with a 10-link synfire chain, every link whose neurons project to the next one shows
up as a subtree of the dendrogram built from the outgoing weights.

Merges (ids, sizes) must be identical; heights agree to 1e-9 relative (FP64 sums in other orders)."""
import numpy as np
import pytest
import torch

import synth
from oracle import ward as ow

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def glm():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1502_04993_gb300 as g
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return g


@pytest.fixture(scope="module")
def ctx(glm):
    c = glm.GLM(0)
    yield c
    c.close()


@pytest.mark.parametrize("by,subset", [("out", None), ("in", None), ("in", "odd")])
def test_ward_matches_oracle(glm, ctx, by, subset):
    n = 150
    W = np.random.default_rng(11).normal(0, 0.3, (n, n)).astype(np.float32)
    sub = np.arange(1, n, 2) if subset == "odd" else None
    Z = ctx.ward(torch.from_numpy(W), by=by, subset=sub)
    Zo = ow.ward_linkage(ow.features(W.astype(np.float64), by, sub))
    assert np.array_equal(Z[:, :2], Zo[:, :2]) and np.array_equal(Z[:, 3], Zo[:, 3])
    assert np.allclose(Z[:, 2], Zo[:, 2], rtol=1e-9, atol=0)
    m = len(Z) + 1
    for k in (2, 5, 17):
        assert np.array_equal(glm.ward_cut(Z, k), ow.cut(Zo, m, k))


def test_synfire_links_are_subtrees(ctx):
    W, _ = synth.network(2000, 1600, 0.05, 0.2, 0.8, 3, w_self=-6.25, syn_groups=10, syn_size=50, w_syn=0.3)
    W = W + np.random.default_rng(4).normal(0, 0.05, W.shape)  # estimation noise of a reconstruction
    Z = ctx.ward(torch.from_numpy(W.astype(np.float32)), by="out")
    m = 2000
    work = {k: {k} for k in range(m)}
    clusters = []  # every subtree of at most 200 neurons (a link has 50)
    for q, (a, b, _, _) in enumerate(Z):
        c = work.pop(int(a)) | work.pop(int(b))
        work[m + q] = c
        if len(c) <= 200:
            clusters.append(c)
    for g in range(9):  # links 1..9 project to the next link; the last one projects nowhere special
        link = set(range(50 * g, 50 * g + 50))
        best = max(len(c & link) / 50 for c in clusters if len(c & link) >= 0.9 * len(c))
        assert best >= 0.9, (g, best)


def test_ward_errors(glm, ctx):
    W = torch.zeros((4, 4))
    with pytest.raises(glm.GLMError):
        ctx.ward(W, by="out", subset=[0, 7])
    with pytest.raises(glm.GLMError):
        glm.ward_cut(np.zeros((3, 4)), 9)
