"""Pins of the oracle's beam-search candidate route (Alg. 3 phases 1-2, Sec. 4.1) against what
fixes it independently: on a complete graph with a queue longer than n the search computes
every distance, so the candidates are the exact C nearest and the beam-candidate build equals
the exact-candidate build; on a sparse K-NN graph the lists are (D, id)-sorted, distinct,
never contain p, and never beat the exact C nearest (they are C points, each at least as far
as the exact i-th)."""
import numpy as np

import oracle
from paper_2510_05975_gb300 import synth


def _complete(n):
    A = np.array([[v for v in range(n) if v != u] for u in range(n)], np.int32)
    return A, np.full(n, n - 1, np.int32)


def test_complete_graph_gives_exact_candidates():
    X = synth.generate("gauss", 120, 6, seed=21)
    n = len(X)
    A, D = _complete(n)
    s = oracle.entry(X)
    ids, ds, cnt = oracle.beam_candidates(X, A, D, s, L=n + 5, C=20)
    exact, eds = oracle.knn(X, 20)
    assert np.all(cnt == 20)
    assert np.array_equal(ids, exact)
    assert np.allclose(ds, eds, rtol=0, atol=0)


def test_beam_build_reduces_to_exact_build():
    X = synth.generate("gauss", 150, 5, seed=22)
    n = len(X)
    A, _ = _complete(n)
    Gb = oracle.build_graph_beam(X, 1.2, 0.0, 8, C=24, K=n - 1, Lb=n + 1, knn_graph=A)
    Ge = oracle.build_graph(X, 1.2, 0.0, 8, 24)
    assert Gb.entry == Ge.entry
    assert np.array_equal(Gb.cand, Ge.cand)
    assert np.array_equal(Gb.fwd, Ge.fwd) and np.array_equal(Gb.adj, Ge.adj)


def test_sparse_graph_candidate_invariants():
    X = synth.generate("gauss", 800, 8, seed=23)
    n = len(X)
    G0 = oracle.knn(X, 10)[0]
    s = oracle.entry(X)
    C = 40
    ids, ds, cnt = oracle.beam_candidates(X, G0, np.full(n, 10, np.int32), s, L=48, C=C)
    _, exact_d = oracle.knn(X, C)
    for p in range(n):
        c = cnt[p]
        row = ids[p, :c]
        assert c > 0 and np.all(ids[p, c:] == -1)
        assert p not in row and len(set(row.tolist())) == c
        keys = list(zip(ds[p, :c].tolist(), row.tolist()))
        assert keys == sorted(keys)
        # the i-th collected point is never closer than the exact i-th nearest
        assert np.all(ds[p, :c] >= exact_d[p, :c] - 1e-12)
