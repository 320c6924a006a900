"""Pins of the matching oracle (correlation of spin images): textbook values
and np.corrcoef."""
import numpy as np

from oracle import match


def _imgs(n, W, seed):
    rng = np.random.default_rng(seed)
    return (rng.poisson(3.0, (n, W, W)) * 65536).astype(np.int32)


def test_correlation_is_numpys_corrcoef():
    a, b = _imgs(7, 8, 1), _imgs(5, 8, 2)
    r = match.correlations(a, b)
    for i in range(7):
        for j in range(5):
            ref = np.corrcoef(a[i].ravel().astype(np.float64), b[j].ravel().astype(np.float64))[0, 1]
            assert abs(r[i, j] - ref) < 1e-12


def test_invariants():
    a = _imgs(4, 16, 3)
    r = match.correlations(a, a)
    np.testing.assert_allclose(np.diag(r), 1.0, atol=1e-12)
    np.testing.assert_allclose(r, r.T, atol=1e-12)
    # a positive affine copy correlates 1, a negative one -1
    b = (a.astype(np.int64) * 3 + 65536 * 5).astype(np.int32)
    np.testing.assert_allclose(np.diag(match.correlations(a, b)), 1.0, atol=1e-12)
    np.testing.assert_allclose(np.diag(match.correlations(a, -a)), -1.0, atol=1e-12)
    assert np.all(np.abs(r) <= 1 + 1e-12)


def test_constant_image_correlates_zero():
    a = _imgs(3, 8, 4)
    c = np.full((1, 8, 8), 65536 * 7, np.int32)
    assert np.all(match.correlations(c, a) == 0.0)
    assert np.all(match.correlations(a, c) == 0.0)


def test_best_matches_order_and_ties():
    a = _imgs(6, 8, 5)
    model = np.concatenate([a[:3], a[:3], _imgs(10, 8, 6)])   # exact duplicates: ties
    idx, r = match.best_matches(a[:3], model, 4)
    for i in range(3):
        assert idx[i, 0] == i and idx[i, 1] == i + 3           # R = 1 twice, smaller index first
        assert np.all(np.diff(r[i]) <= 0)
