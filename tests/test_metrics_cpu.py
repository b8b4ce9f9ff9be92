"""Clustering accuracy of Sec. 3.2 (Eq. 3-4): the oracle pinned against
brute-force pair counts, closed cases (a pure topic, an even spread, at most
one member) and invariances, and the library's histogram form against the
oracle."""
import itertools

import numpy as np
import pytest

import oracle
from paper_1510_05237_gb300 import metrics


def brute_same_pairs(labels):
    return sum(1 for a, b in itertools.combinations(labels, 2) if a == b)


@pytest.mark.parametrize("n_j", [1, 2, 3, 5, 7])
def test_alpha_counts_the_pairs_of_an_even_spread(n_j):
    """alpha of Eq. 4 is the same-class pair count of the most even spread:
    an even spread therefore scores 0, checked against brute-force counts."""
    for n_d in range(2, 40):
        labels = np.arange(n_d) % n_j          # as even as it gets
        V = np.ones((n_d, 1))
        acc = oracle.topic_accuracy(V, labels, n_j)
        q, r = divmod(n_d, n_j)
        alpha = brute_same_pairs(labels)
        beta = n_d * (n_d - 1) // 2
        assert alpha == q * n_j * (q - 1) // 2 + q * r   # Eq. 4's alpha, exactly
        if beta != alpha:
            assert acc[0] == pytest.approx(0.0, abs=1e-15)
        else:
            assert acc[0] == 1.0


def test_pure_topic_and_small_topics_score_one():
    labels = np.array([3, 3, 3, 1, 0, 2, 3])
    V = np.zeros((7, 3))
    V[[0, 1, 2, 6], 0] = 0.5       # four members, all of class 3
    V[4, 1] = 1.0                  # one member
    acc = oracle.topic_accuracy(V, labels, 4)   # column 2: no member
    np.testing.assert_array_equal(acc, [1.0, 1.0, 1.0])


def test_random_topics_match_the_definition_by_brute_force():
    rng = np.random.default_rng(11)
    for trial in range(20):
        m, k, n_j = int(rng.integers(2, 60)), int(rng.integers(1, 6)), int(rng.integers(2, 6))
        labels = rng.integers(0, n_j, size=m)
        V = rng.random((m, k)) * (rng.random((m, k)) < 0.4)
        acc = oracle.topic_accuracy(V, labels, n_j)
        for c in range(k):
            mem = labels[V[:, c] != 0]
            n_d = len(mem)
            if n_d <= 1:
                assert acc[c] == 1.0
                continue
            same = brute_same_pairs(mem)
            q, r = divmod(n_d, n_j)
            alpha = q * (n_j * (q - 1) / 2 + r)
            beta = n_d * (n_d - 1) / 2
            assert acc[c] == pytest.approx((same - alpha) / (beta - alpha), abs=1e-12)
            assert acc[c] <= 1.0 + 1e-12


def test_accuracy_ignores_values_and_class_names():
    """Only the support of V and the partition of the documents matter: the
    values can be rescaled and the classes renamed."""
    rng = np.random.default_rng(5)
    labels = rng.integers(0, 4, size=50)
    V = rng.random((50, 3)) * (rng.random((50, 3)) < 0.5)
    perm = np.array([2, 0, 3, 1])
    a = oracle.topic_accuracy(V, labels, 4)
    np.testing.assert_array_equal(a, oracle.topic_accuracy(7.0 * V, perm[labels], 4))


def test_library_form_matches_the_oracle():
    rng = np.random.default_rng(3)
    for trial in range(10):
        m, k, n_j = int(rng.integers(2, 400)), int(rng.integers(1, 9)), int(rng.integers(1, 9))
        labels = rng.integers(0, n_j, size=m)
        V = rng.random((m, k)) * (rng.random((m, k)) < 0.3)
        np.testing.assert_allclose(metrics.topic_accuracy(V, labels, n_j),
                                   oracle.topic_accuracy(V, labels, n_j), rtol=0, atol=1e-12)


def test_library_rejects_bad_labels():
    with pytest.raises(ValueError):
        metrics.topic_accuracy(np.ones((3, 1)), np.array([0, 1, 2]), 2)


def test_factor_dense_round_trip():
    rng = np.random.default_rng(8)
    F = rng.random((30, 4)) * (rng.random((30, 4)) < 0.3)
    colptr = np.concatenate([[0], np.cumsum((F != 0).sum(axis=0))])
    rowidx = np.concatenate([np.nonzero(F[:, c])[0] for c in range(4)])
    vals = np.concatenate([F[F[:, c] != 0, c] for c in range(4)])
    np.testing.assert_array_equal(metrics.factor_dense((colptr, rowidx, vals), 30, 4), F)
