"""Host arithmetic of the studies (CPU only).

The label-agreement measure of the recursion study: the adjusted Rand index
from the contingency table, checked against a brute-force count over all
pixel pairs and, where scikit-learn is installed, against its
implementation.  The screen-error study: its exact keys against rationals
and the two-pixel closed form, and its error bound, which a binary32 Gram
must meet and a perturbed Gram must break."""
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


def _groups(seed, R, B, nmax):
    """R regions of random sizes 1..nmax with integer pixel sums."""
    rng = np.random.default_rng(seed)
    n = rng.integers(1, nmax + 1, R)
    base = rng.integers(500, 9000, (8, B))
    S = np.stack([rng.integers(0, 200, (k, B)).sum(axis=0) + k * base[rng.integers(0, 8)] for k in n])
    return S.astype(np.int64), n.astype(np.int64)


def test_exact_keys_against_rationals():
    from fractions import Fraction
    from paper_2106_12942_b300.studies import exact_keys
    S, n = _groups(3, 9, 5, 40)
    K = exact_keys(S, n)
    for i in range(9):
        for j in range(9):
            mi = [Fraction(int(v), int(n[i])) for v in S[i]]
            mj = [Fraction(int(v), int(n[j])) for v in S[j]]
            ref = Fraction(int(n[i] * n[j]), int(n[i] + n[j])) * sum((a - b) ** 2 for a, b in zip(mi, mj))
            assert abs(K[i, j] - float(ref)) <= 1e-13 * float(ref)
    p = np.array([[3, 10, 7], [0, 4, 1]], np.int64)                # two pixels: K = |p - q|^2 / 2
    assert exact_keys(p, np.ones(2, np.int64))[0, 1] == 0.5 * (9 + 36 + 36)


def _f32_gram(Xh):
    x = Xh.float().numpy()
    return x @ x.T                                                    # binary32 accumulation


@pytest.mark.parametrize("precision", [1, 2])
def test_screen_error_bound_holds_for_binary32_gram(precision):
    pytest.importorskip("torch")
    from paper_2106_12942_b300.studies import screen_error_of
    S, n = _groups(7 + precision, 300, 200, 500)
    r = screen_error_of(S, n, precision, _f32_gram)
    assert r["pairs"] == 300 * 299 // 2
    assert 0.0 < r["max_err_over_bound"] <= 1.0
    assert r["max_rel_err"] > 0.0


def test_screen_error_bound_catches_a_perturbed_gram():
    pytest.importorskip("torch")
    from paper_2106_12942_b300.studies import screen_error_of
    S, n = _groups(11, 200, 200, 500)
    bad = lambda Xh: _f32_gram(Xh) * (1.0 + 1e-3 * (1 - np.eye(Xh.shape[0])))   # off-diagonal 0.1 % high
    assert screen_error_of(S, n, 1, bad)["max_err_over_bound"] > 1.0
    drop = lambda Xh: _f32_gram(Xh[:, :-40].contiguous())             # a band block left out
    assert screen_error_of(S, n, 1, drop)["max_err_over_bound"] > 1.0


def test_screen_rows_scale_keeps_fp16_finite():
    torch = pytest.importorskip("torch")
    from paper_2106_12942_b300.studies import screen_rows
    n = np.array([1, 3, 7, 1], np.int64)
    S = np.stack([np.full(5, 65535) * n[0], np.zeros(5, np.int64), np.full(5, 65535) * n[2], np.full(5, 17)])
    x32, s, xs = screen_rows(S, n, 32)
    assert np.abs(x32).max() < 2.0 ** 15 and s >= 1
    assert torch.isfinite(torch.from_numpy(x32).half()).all()
    assert np.allclose(x32[:, :5], xs, rtol=2.0 ** -22, atol=0)
    assert np.all(x32[:, 5:] == 0)
