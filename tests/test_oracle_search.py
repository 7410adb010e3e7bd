"""Pins for the oracle's beam search (Alg. 1)."""
import numpy as np

import oracle
from paper_2510_05975_gb300 import synth


def test_path_graph_greedy():
    X = np.arange(10, dtype=np.float32)[:, None]
    adj = np.full((10, 2), -1, np.int32)
    deg = np.zeros(10, np.int32)
    for i in range(10):
        nb = [j for j in (i - 1, i + 1) if 0 <= j < 10]
        adj[i, : len(nb)] = nb
        deg[i] = len(nb)
    ids, ds, ndc, hops = oracle.search(X, adj, deg, 0, np.array([[9.3]], np.float32), 1, 1)
    assert ids[0, 0] == 9 and hops[0] == 10 and ndc[0] == 10
    assert abs(ds[0, 0] - 0.3) < 1e-6


def test_star_graph_queue():
    # centre 0 linked to 1..6 only: one hop explores everything reachable.
    X = np.array([[0, 0], [1, 0], [2, 0], [3, 0], [0, 1], [0, 2], [0, 3]], np.float32)
    adj = np.full((7, 6), -1, np.int32)
    deg = np.zeros(7, np.int32)
    adj[0] = [1, 2, 3, 4, 5, 6]
    deg[0] = 6
    ids, ds, ndc, hops = oracle.search(X, adj, deg, 0, np.array([[2.9, 0.1]], np.float32), 3, 7)
    assert ids[0].tolist() == [3, 2, 1]
    assert ndc[0] == 7 and hops[0] == 7


def test_large_queue_equals_brute_force():
    X = synth.generate("gauss", 400, 6, seed=21)
    Q = synth.generate("gauss", 20, 6, seed=22)
    G = oracle.build_graph(X, 1.2, 0.0, 12, 30)
    ids, ds, ndc, hops = oracle.search(X, G.adj, G.deg, G.entry, Q, 10, 400)
    ref = np.argsort(np.linalg.norm(Q[:, None].astype(np.float64) - X[None].astype(np.float64), axis=2), axis=1)[:, :10]
    # every point reachable from the entry ends in Q when L >= n
    reach = _reachable(G)
    if len(reach) == len(X):
        assert np.array_equal(ids, ref)
        assert np.all(ndc == len(X))


def _reachable(G):
    seen, stack = {G.entry}, [G.entry]
    while stack:
        u = stack.pop()
        for v in G.out(u):
            if int(v) not in seen:
                seen.add(int(v))
                stack.append(int(v))
    return seen


def test_recall_definition():
    assert oracle.recall([[1, 2, 3]], [[3, 2, 9]]) == 2 / 3


def _graph(lists, n):
    R = max(1, max(len(v) for v in lists.values()))
    adj = np.full((n, R), -1, np.int32)
    deg = np.zeros(n, np.int32)
    for u, nb in lists.items():
        adj[u, : len(nb)] = nb
        deg[u] = len(nb)
    return adj, deg


def test_hop_vertex_is_nearest_unexplored():
    # Worked by hand (Alg. 1, L = 2, q = 3.0 on a line): exploring 0 leaves Q = [2 (1.5),
    # 1 (2.0)]; the nearest unexplored is 2, whose neighbour 3 (0.4) evicts 1 before 1 is
    # ever explored, so 4 (0.05, reachable only through 1) is never seen.
    X = np.array([[0.0], [1.0], [1.5], [2.6], [3.05]], np.float32)
    adj, deg = _graph({0: [1, 2], 1: [4], 2: [3]}, 5)
    ids, ds, ndc, hops = oracle.search(X, adj, deg, 0, np.array([[3.0]], np.float32), 1, 2)
    assert ids[0, 0] == 3 and hops[0] == 3 and ndc[0] == 4


def test_queue_ties_keep_smaller_ids():
    # four neighbours at exactly distance 1 from q, inserted in descending id order; with
    # L = 2 the (D, id) order keeps ids 1 and 2.
    X = np.array([[5, 5], [1, 0], [-1, 0], [0, 1], [0, -1]], np.float32)
    adj, deg = _graph({0: [4, 3, 2, 1]}, 5)
    ids, ds, ndc, hops = oracle.search(X, adj, deg, 0, np.array([[0, 0]], np.float32), 2, 2)
    assert ids[0].tolist() == [1, 2]
