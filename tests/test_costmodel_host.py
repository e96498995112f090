"""Host-side logic of the cost-model choosers (no GPU): the per-region
capacity rule and the non-negative least squares that fits unit costs of
the logged work to the logged phase times."""
import numpy as np
import pytest

from paper_1411_3212_gb300.costmodel import nonneg_lstsq, region_caps


def test_region_caps_rule():
    """Per-region capacities of the cost-model chooser: 2^(a + b log2 d_r)
    with d_r the region's density over the mean; empty regions take 2^a."""
    counts = np.array([300, 100, 0, 0])            # densities 3, 1, -, - (mean 1 per region)
    np.testing.assert_array_equal(region_caps(counts, 1, 7, 0.0), [128] * 4)
    np.testing.assert_array_equal(region_caps(counts, 1, 7, 1.0), [384, 128, 128, 128])
    np.testing.assert_array_equal(region_caps(counts, 1, 7, -1.0), [43, 128, 128, 128])
    np.testing.assert_array_equal(region_caps(counts, 1, 14, 1.0), [16384, 16384, 16384, 16384])
    np.testing.assert_array_equal(region_caps([0, 0, 0, 0], 1, 3, 0.5), [8] * 4)
    big = np.zeros(16, np.int64)
    big[5] = 10 ** 6
    big[6] = 1
    c = region_caps(big, 2, 4, -1.0)
    assert c[5] == 1 and c[6] == 16384 and c[0] == 16
    with pytest.raises(ValueError):
        region_caps(counts, 2, 7, 0.0)


def test_nonneg_lstsq_recovers_nonnegative_coefficients():
    rng = np.random.default_rng(1)
    A = rng.uniform(0, 1, (40, 5))
    x = np.array([2.0, 0.0, 0.5, 3.0, 0.0])
    np.testing.assert_allclose(nonneg_lstsq(A, A @ x), x, atol=1e-9)
    # a target that ordinary least squares fits with a negative weight
    b = A @ np.array([1.0, 0.0, 0.0, 0.0, 0.0]) - 0.3 * A[:, 1]
    sol = nonneg_lstsq(A, b)
    assert np.all(sol >= 0) and sol[1] == 0.0
    # the kept columns are the least-squares fit on those columns alone
    keep = sol > 0
    ls, *_ = np.linalg.lstsq(A[:, keep], b, rcond=None)
    np.testing.assert_allclose(sol[keep], ls, atol=1e-9)
