"""The label-agreement measure of the recursion study (CPU only): the
adjusted Rand index from the contingency table, checked against a brute-force
count over all pixel pairs and, where scikit-learn is installed, against its
implementation."""
import numpy as np
import pytest

from paper_2106_12942_b300.studies import adjusted_rand_index


def _ari_brute(a, b):
    a = a.ravel()
    b = b.ravel()
    n = a.size
    iu = np.triu_indices(n, 1)
    sa = (a[:, None] == a[None, :])[iu]
    sb = (b[:, None] == b[None, :])[iu]
    pairs = n * (n - 1) / 2.0
    both, na, nb = float(np.sum(sa & sb)), float(np.sum(sa)), float(np.sum(sb))
    expected = na * nb / pairs
    return (both - expected) / (0.5 * (na + nb) - expected)


def test_ari_matches_pair_count():
    rng = np.random.default_rng(5)
    for _ in range(12):
        a = rng.integers(1, 7, (18, 20))
        b = a.copy()
        flip = rng.random(a.shape) < rng.random()
        b[flip] = rng.integers(1, 7, int(flip.sum()))
        assert abs(adjusted_rand_index(a, b) - _ari_brute(a, b)) < 1e-12


def test_ari_matches_sklearn():
    metrics = pytest.importorskip("sklearn.metrics")
    rng = np.random.default_rng(9)
    a = rng.integers(1, 9, (30, 40))
    b = np.where(rng.random(a.shape) < 0.3, rng.integers(1, 9, a.shape), a)
    assert abs(adjusted_rand_index(a, b) - metrics.adjusted_rand_score(a.ravel(), b.ravel())) < 1e-12


def test_ari_ignores_masked_and_is_label_invariant():
    rng = np.random.default_rng(6)
    a = rng.integers(1, 5, (20, 20))
    perm = np.array([0, 3, 1, 4, 2])
    assert adjusted_rand_index(a, perm[a]) == 1.0
    b = a.copy()
    b[0, :] = 0                                    # masked pixels do not count
    assert adjusted_rand_index(a, b) == 1.0
