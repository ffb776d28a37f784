"""The label-agreement measure of the recursion study, checked against
scikit-learn's adjusted Rand index (CPU only)."""
import numpy as np
from sklearn.metrics import adjusted_rand_score

from paper_2106_12942_b300.studies import adjusted_rand_index


def test_ari_matches_sklearn():
    rng = np.random.default_rng(5)
    for _ in range(20):
        a = rng.integers(1, 9, (30, 40))
        b = a.copy()
        flip = rng.random(a.shape) < rng.random()
        b[flip] = rng.integers(1, 9, int(flip.sum()))
        assert abs(adjusted_rand_index(a, b) - adjusted_rand_score(a.ravel(), b.ravel())) < 1e-12


def test_ari_ignores_masked_and_is_label_invariant():
    rng = np.random.default_rng(6)
    a = rng.integers(1, 5, (20, 20))
    perm = np.array([0, 3, 1, 4, 2])
    assert adjusted_rand_index(a, perm[a]) == 1.0
    b = a.copy()
    b[0, :] = 0                                    # masked pixels do not count
    assert adjusted_rand_index(a, b) == 1.0
