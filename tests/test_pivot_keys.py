"""The leaf kernel's pivot search compares the bit patterns of |a_ik| as
unsigned integers (NaN clamped to +inf) instead of the doubles themselves.
That is the same order: for non-negative IEEE doubles the bit patterns
increase with the value, across zero, subnormals, normals and infinity.
Checked here on the host with numpy's view of the same bits."""
import numpy as np

INF_BITS = np.uint64(0x7FF0000000000000)


def key(a):
    mag = np.abs(a).view(np.uint64) & np.uint64(0x7FFFFFFFFFFFFFFF)
    return np.minimum(mag, INF_BITS)


def test_bit_order_is_value_order():
    rng = np.random.default_rng(7)
    vals = np.concatenate([
        rng.uniform(0, 1, 2000), rng.uniform(0, 1e300, 500), 2.0 ** rng.integers(-1074, 1023, 500).astype(float),
        np.array([0.0, -0.0, 5e-324, 2.2250738585072014e-308, 1.0, np.inf, -np.inf, 1.7976931348623157e308]),
        -rng.uniform(0, 10, 500),
    ])
    k = key(vals)
    mags = np.abs(vals)
    order_v = np.lexsort((np.arange(len(vals)), mags))
    order_k = np.lexsort((np.arange(len(vals)), k))
    np.testing.assert_array_equal(mags[order_v], mags[order_k])
    # equal keys exactly when equal magnitudes (-0.0 and 0.0 share a key)
    i, j = rng.integers(0, len(vals), (2, 5000))
    assert np.array_equal(k[i] == k[j], mags[i] == mags[j])
    assert np.array_equal(k[i] < k[j], mags[i] < mags[j])


def test_nan_is_clamped_to_infinity():
    nans = np.array([np.nan, -np.nan, np.float64("nan")]).astype(np.float64)
    payload = np.array([0x7FF8000000000001, 0xFFF0000000000001], dtype=np.uint64).view(np.float64)
    k = key(np.concatenate([nans, payload]))
    assert (k == INF_BITS).all()
    assert key(np.array([np.inf]))[0] == INF_BITS


def test_argmax_rule_matches_oracle_pivot_rule():
    """Largest key, lowest position on ties: the rule of the oracle's
    Gauss-Jordan (largest |a_ik|, lowest position)."""
    rng = np.random.default_rng(11)
    for _ in range(200):
        col = rng.choice([0.0, 0.5, -0.5, 1.0, -1.0, 2.0], size=rng.integers(1, 40))
        pos = rng.permutation(len(col))
        k = key(col)
        best = max(range(len(col)), key=lambda r: (k[r], -pos[r]))
        want = max(range(len(col)), key=lambda r: (abs(col[r]), -pos[r]))
        assert best == want
