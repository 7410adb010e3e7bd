"""Pins for the oracle's canonical distance and exact candidate lists (Sec. 2.1, Alg. 3)."""
import math

import numpy as np
import pytest

import oracle
from paper_2510_05975_gb300 import synth


def test_pythagorean_triple_is_exact():
    assert oracle.dist([0.0, 0.0], [3.0, 4.0]) == 5.0
    assert oracle.sqdist([1.0, 2.0, 2.0], [0.0, 0.0, 0.0]) == 9.0


def test_sum_is_left_to_right():
    # squares 2^54, 1, 1, 1, 1: a left-to-right sum absorbs every 1 (ulp(2^54) = 4), a
    # right-to-left or pairwise sum would give 2^54 + 4.
    x = np.array([2.0 ** 27, 1, 1, 1, 1], np.float32)
    y = np.zeros(5, np.float32)
    assert oracle.sqdist(x, y) == 2.0 ** 54
    assert oracle.sqdist(x[::-1].copy(), y) == 2.0 ** 54 + 4


def test_matches_library_norm():
    rng = np.random.default_rng(5)
    for d in (1, 7, 32, 960):
        x = rng.standard_normal(d).astype(np.float32)
        y = rng.standard_normal(d).astype(np.float32)
        ref = float(np.linalg.norm(x.astype(np.float64) - y.astype(np.float64)))
        assert abs(oracle.dist(x, y) - ref) <= 1e-14 * ref


def test_fp16_widening_is_exact():
    h = np.array([0.1, -3.5, 65504.0], np.float16)
    assert oracle.sqdist(h, np.zeros(3, np.float16)) == sum(float(v) ** 2 for v in h.astype(np.float64))


def _brute_lists(X, L):
    """Independent reference: numpy distances, lexsort on (distance, id)."""
    X64 = X.astype(np.float64)
    out = []
    for i in range(X.shape[0]):
        dd = np.linalg.norm(X64 - X64[i], axis=1)
        dd[i] = np.inf
        order = np.lexsort((np.arange(X.shape[0]), dd))
        out.append(order[:L])
    return np.array(out)


def test_knn_matches_brute_force_continuous():
    X = synth.generate("gauss", 300, 16, seed=11)
    ids, ds = oracle.knn(X, 20)
    assert np.array_equal(ids, _brute_lists(X, 20))
    assert np.all(np.diff(ds, axis=1) >= 0)


def test_knn_ties_break_by_id():
    # integer grid on a line: exact ties everywhere, squared distances are integers
    X = np.array([[0], [2], [-1], [1], [-2], [3], [1]], np.float32)
    ids, ds = oracle.knn(X, 6)
    for i in range(len(X)):
        keyed = sorted((int(round((X[j, 0] - X[i, 0]) ** 2)), j) for j in range(len(X)) if j != i)
        assert ids[i].tolist() == [j for _, j in keyed[:6]]
    # the duplicate (ids 3 and 6 at x = 1) stays a candidate: excluded by id, not by value
    assert ids[3][0] == 6 and ds[3][0] == 0.0


def test_knn_queries_and_padding():
    X = synth.generate("gauss", 50, 8, seed=3)
    Q = synth.generate("gauss", 5, 8, seed=4)
    ids, ds = oracle.knn(X, 60, rows=Q)
    assert np.all(ids[:, 50:] == -1) and np.all(np.isinf(ds[:, 50:]))
    ref = np.argsort(np.linalg.norm(Q[:, None, :].astype(np.float64) - X[None].astype(np.float64), axis=2), axis=1)
    assert np.array_equal(ids[:, :50], ref)


def test_centroid_and_entry():
    X = synth.generate("sift", 2000, 24, seed=2)
    c = oracle.centroid(X)
    assert np.allclose(c, X.astype(np.float64).mean(axis=0), rtol=1e-13, atol=0)
    dd = np.linalg.norm(X.astype(np.float64) - X.astype(np.float64).mean(axis=0), axis=1)
    best = np.flatnonzero(dd <= dd.min() * (1 + 1e-12))
    assert oracle.entry(X) == int(best.min())
