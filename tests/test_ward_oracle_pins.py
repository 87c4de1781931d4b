"""Pins of the Ward clustering oracle (oracle.ward) to results it does not compute itself.

* SciPy's hierarchical clustering (scipy.cluster.hierarchy.linkage, method 'ward', the paper's tool,
  Sec. 3.4.2), an independent implementation by nearest-neighbour chains and the Lance-Williams update:
  the same merges, heights to rounding, sizes; and the same partitions when cut into k clusters.
* Ward's identity: every merge raises the within-cluster sum of squares by height^2 / 2, so the heights
  add up to the total sum of squares about the grand mean.
* Planted structure: columns of W drawn from three well-separated groups come back as those groups.
"""
import numpy as np
import pytest

from oracle import ward

hier = pytest.importorskip("scipy.cluster.hierarchy")


def same_partition(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return all(len(set(b[a == v])) == 1 for v in set(a)) and all(len(set(a[b == v])) == 1 for v in set(b))


@pytest.mark.parametrize("seed,n,f", [(0, 40, 7), (1, 25, 60), (2, 60, 3)])
def test_matches_scipy(seed, n, f):
    X = np.random.default_rng(seed).normal(size=(n, f))
    Z = ward.ward_linkage(X)
    Zs = hier.linkage(X, method="ward")
    assert np.array_equal(Z[:, :2], Zs[:, :2])
    assert np.allclose(Z[:, 2], Zs[:, 2], rtol=1e-11, atol=0)
    assert np.array_equal(Z[:, 3], Zs[:, 3])
    for k in (2, 3, 7):
        assert same_partition(ward.cut(Z, n, k), hier.fcluster(Zs, k, criterion="maxclust"))


def test_heights_add_up_to_the_sum_of_squares():
    X = np.random.default_rng(4).normal(size=(30, 5)) * [1, 2, 3, 4, 5]
    Z = ward.ward_linkage(X)
    assert (Z[:, 2] ** 2 / 2).sum() == pytest.approx(((X - X.mean(axis=0)) ** 2).sum(), rel=1e-12)
    assert np.all(np.diff(Z[:, 2]) >= 0)  # Ward merges never come down


def test_planted_column_groups():
    rng = np.random.default_rng(5)
    n = 45
    W = rng.normal(0, 0.05, (n, n))
    groups = np.repeat([0, 1, 2], 15)
    for g, v in enumerate([0.0, 0.8, -1.0]):
        W[:, groups == g] += v * (rng.random((n, 15)) < 0.5)
    labels = ward.cut(ward.ward_linkage(ward.features(W, "out")), n, 3)
    assert same_partition(labels, groups)
