"""Pins of the oracle's inner-product augmentation (the library's CNG_IP metric) against what
the algebra fixes: Euclidean order on augmented rows is decreasing inner-product order, every
augmented row has norm M, and the squared distance has the closed form |q|^2 + M^2 - 2 <q, x>."""
import numpy as np

import oracle


def _data(seed, n=400, d=12):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, d)) * rng.uniform(0.2, 3.0, (n, 1))  # rows of varied norm
    Q = rng.standard_normal((25, d)) * 1.7
    return X.astype(np.float32), Q.astype(np.float32)


def test_augmented_rows_have_norm_M():
    X, _ = _data(1)
    Xa, M2 = oracle.mips_augment(X)
    assert Xa.shape == (X.shape[0], X.shape[1] + 1) and Xa.dtype == np.float32
    assert np.array_equal(Xa[:, :-1], X)
    n2 = (Xa.astype(np.float64) ** 2).sum(axis=1)
    assert np.allclose(n2, M2, rtol=1e-6)
    assert np.all(Xa[:, -1] >= 0)
    assert Xa[np.argmax((X.astype(np.float64) ** 2).sum(axis=1)), -1] == 0.0


def test_euclidean_order_is_inner_product_order():
    X, Q = _data(2)
    Xa, M2 = oracle.mips_augment(X)
    Qa = oracle.mips_queries(Q)
    assert np.array_equal(Qa[:, :-1], Q) and np.all(Qa[:, -1] == 0)
    ip = Q.astype(np.float64) @ X.astype(np.float64).T
    d2 = ((Qa.astype(np.float64)[:, None, :] - Xa.astype(np.float64)[None, :, :]) ** 2).sum(-1)
    closed = (Q.astype(np.float64) ** 2).sum(1)[:, None] + M2 - 2 * ip
    assert np.allclose(d2, closed, rtol=1e-5, atol=1e-4)
    for i in range(len(Q)):
        assert np.array_equal(np.argsort(d2[i], kind="stable")[:10], np.argsort(-ip[i], kind="stable")[:10])
    # the oracle's exact k-NN on augmented rows returns the top inner products
    ids, _ = oracle.knn(Xa, 10, rows=Qa)
    assert np.array_equal(ids, np.argsort(-ip, axis=1, kind="stable")[:, :10])


def test_norms_are_sequential_fp64_sums():
    # integer rows: every partial sum is exact, so M^2 is the exact largest squared norm
    rng = np.random.default_rng(3)
    X = rng.integers(-40, 41, (200, 30)).astype(np.float32)
    _, M2 = oracle.mips_augment(X)
    assert M2 == max(int((r.astype(np.int64) ** 2).sum()) for r in X)
