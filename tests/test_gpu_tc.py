"""The tensor-core contraction behind the spectral screen (TMA + tcgen05,
FP16/BF16 operands, FP32 accumulation) against the exact product.

The screen's soundness rests on |g - <x_i, x_j>| <= gamma * sum_b |x_ib x_jb|
with gamma = Bpad * 2^-22 (products exact in FP32, one rounding per
addition, a factor 2 of margin); this test measures that ratio and also
catches any layout error (swizzle, descriptor, transposition), which would
produce errors of the size of the entries themselves."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_2106_12942_b300 as P
    return P


@pytest.mark.parametrize("cta_pair", [0, 1])
@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("rows,bpad", [(128, 64), (256, 128), (384, 256), (128, 448), (256, 224), (128, 32), (256, 96),
                                       (640, 224)])
def test_gram_matches_exact_product(P, precision, rows, bpad, cta_pair):
    """One-CTA form and CTA-pair form (two CTAs share each 256x256 tile; a
    wrong operand split or column order shows as errors of the size of the
    entries)."""
    import torch
    rng = np.random.default_rng(rows * 7 + bpad + precision)
    X = rng.normal(0, 1000, (rows, bpad))
    X[:, bpad - 16:] = 0.0                       # zero padding as in the operand rows
    X[rng.random(rows) < 0.1] *= 1e-3            # mixed magnitudes
    dt = torch.float16 if precision == 1 else torch.bfloat16
    Xt = torch.tensor(X, dtype=dt, device="cuda")
    G = P.gram_tc(Xt, precision=precision, cta_pair=cta_pair).cpu().numpy().astype(np.float64)
    Xq = Xt.float().cpu().numpy().astype(np.float64)          # the values the tensor cores saw
    exact = Xq @ Xq.T                                           # products and sums exact in float64 here
    absum = np.abs(Xq) @ np.abs(Xq).T
    gamma = bpad * 2.0 ** -22
    ratio = np.abs(G - exact) / np.maximum(gamma * absum, 1e-300)
    assert np.all(np.isfinite(G))
    assert ratio.max() <= 1.0, ratio.max()
    # sanity of the layout: the error is tiny relative to the entries
    assert np.abs(G - exact).max() <= 1e-3 * np.abs(exact).max()


def test_gram_rejects_bad_shapes(P):
    import torch
    with pytest.raises(P.RHSEGError):
        P.gram_tc(torch.zeros(100, 64, dtype=torch.float16, device="cuda"))
    with pytest.raises(P.RHSEGError):
        P.gram_tc(torch.zeros(128, 40, dtype=torch.float16, device="cuda"))
    with pytest.raises(P.RHSEGError):
        P.gram_tc(torch.zeros(128, 48, dtype=torch.float16, device="cuda"))
    with pytest.raises(P.RHSEGError):
        P.gram_tc(torch.zeros(128, 64, dtype=torch.float16, device="cuda"), cta_pair=2)


@pytest.mark.parametrize("precision", [1, 2])
def test_screen_error_on_region_means_within_bound(P, precision):
    """The screen arithmetic's error on real operands (the root-level regions
    of the 145x145x200 run and 2048 random pixels of its cube), through the
    tensor-core Gram, stays within the bound the reject test relies on."""
    from paper_2106_12942_b300.studies import screen_error
    for r in screen_error(precision=precision):
        assert r["pairs"] > 1000, r
        assert r["max_err_over_bound"] <= 1.0, r
        print(r)
