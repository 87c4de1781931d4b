"""Host-side helpers that need no GPU: splitting a recording for cross-validation."""
import numpy as np

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
