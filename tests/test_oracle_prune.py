"""Pins for the oracle's pruning (Def. 2 / Eq. 1, Alg. 2, Alg. 4) and construction (Alg. 3)."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2510_05975_gb300 import synth


def _load(golden_dir, name):
    with open(os.path.join(golden_dir, name)) as f:
        return json.load(f)


def test_hand_worked_2d_example(golden_dir):
    g = _load(golden_dir, "prune_2d.json")
    names = list(g["points"])
    X = np.array([g["p"]] + [g["points"][k] for k in names], np.float32)
    V = np.arange(1, len(names) + 1, dtype=np.int32)[::-1].copy()  # any input order
    for case in g["cases"]:
        S = oracle.prune(X, 0, V, case["alpha"], case["tau"], case["R"])
        assert [names[i - 1] for i in S] == case["kept"], case["why"]
    a = g["adaptive"]
    S, alpha = oracle.prune_adaptive(X, 0, V, a["alpha0"], a["alpha_max"], a["dalpha"], a["tau"], a["R"])
    assert [names[i - 1] for i in S] == a["kept"], a["why"]
    assert alpha == pytest.approx(a["alpha"], abs=1e-12)


def test_adaptive_reaches_alpha_max_exactly():
    # 0.9 + 14 * 0.05 accumulated by repeated addition exceeds 1.6; the oracle must still try 1.6.
    X = np.array([[0, 0], [1, 0], [1.2, 0.1], [1.3, -0.1]], np.float32)
    S, alpha = oracle.prune_adaptive(X, 0, [1, 2, 3], 0.9, 1.6, 0.05, 0.0, 100)
    assert alpha == pytest.approx(1.6, abs=1e-12)


def test_equality_keeps_the_candidate():
    # Eq. 1 is strict: D(p,u) == alpha * D(u,v) + (alpha+1) tau keeps u.
    # p=0, v at 1, u at 2 on a line: D(p,u) = 2, D(u,v) = 1; alpha = 2, tau = 0 -> equality.
    X = np.array([[0.0], [1.0], [2.0]], np.float32)
    assert oracle.prune(X, 0, [1, 2], 2.0, 0.0, 10).tolist() == [1, 2]
    assert oracle.prune(X, 0, [1, 2], 1.5, 0.0, 10).tolist() == [1]


def test_merge_hand_worked(golden_dir):
    g = _load(golden_dir, "merge_2d.json")
    X = np.array(g["points"], np.float32)
    for case in g["cases"]:
        G = oracle.build_graph(X, g["alpha"], g["tau"], case["R"], g["L"])
        assert G.cand.tolist() == g["cand"]
        assert [G.fwd[p, : G.fdeg[p]].tolist() for p in range(len(X))] == g["fwd"]
        assert [G.adj3[p, : G.deg3[p]].tolist() for p in range(len(X))] == case["adj"]
        assert [G.out(p).tolist() for p in range(len(X))] == case["adj4"]


def _alpha_cg(X, alpha, tau):
    """alpha-CG of Def. 3: pruning over P \\ {p}, no degree bound."""
    n = len(X)
    return [oracle.prune(X, p, np.array([u for u in range(n) if u != p], np.int32), alpha, tau, n)
            for p in range(n)]


def _scaled_points(n, d, seed):
    """Random points scaled so the minimum pairwise distance is exactly 1 (Sec. 2.1)."""
    X = synth.generate("gauss", n, d, seed=seed).astype(np.float64)
    D = np.linalg.norm(X[:, None] - X[None], axis=2)
    D[np.diag_indices(n)] = np.inf
    return (X / D.min()).astype(np.float32)


@pytest.mark.parametrize("alpha,tau,seed", [(1.2, 1.0, 1), (1.5, 2.0, 2), (1.1, 1.5, 3)])
def test_lemma1_alpha_reducible_and_lemma3_hops(alpha, tau, seed):
    """Lemma 1 and Lemma 3 on the alpha-CG: for q with D(q, v*) <= tau every p != v* has v*
    or a neighbour p' with D(p', q) <= D(p, q) / alpha, and greedy routing (L = 1) reaches v*
    within log_alpha(4 Delta) + 2 hop vertices."""
    n, d = 120, 3
    X = _scaled_points(n, d, seed)
    G = _alpha_cg(X, alpha, tau)
    deg = np.array([len(s) for s in G], np.int32)
    adj = np.full((n, max(deg)), -1, np.int32)
    for p, s in enumerate(G):
        adj[p, : len(s)] = s
    X64 = X.astype(np.float64)
    diam = max(np.linalg.norm(X64[i] - X64, axis=1).max() for i in range(n))
    bound = math.log(4 * diam) / math.log(alpha) + 2
    rng = np.random.default_rng(seed)
    checked = 0
    for _ in range(60):
        v = int(rng.integers(n))
        off = rng.standard_normal(d)
        q = X64[v] + off / np.linalg.norm(off) * rng.uniform(0, tau)
        dq = np.linalg.norm(X64 - q, axis=1)
        vstar = int(np.argmin(dq))
        if dq[vstar] > tau:
            continue
        checked += 1
        for p in range(n):
            if p == vstar:
                continue
            nb = G[p]
            assert vstar in nb or any(dq[u] <= dq[p] / alpha for u in nb)
        for s in rng.integers(0, n, size=5):
            ids, _, _, hops = oracle.search(X, adj, deg, int(s), q[None].astype(np.float32), 1, 1)
            assert ids[0, 0] == vstar
            assert hops[0] <= bound
    assert checked >= 20


@pytest.mark.parametrize("alpha,tau", [(1.2, 0.0), (1.3, 0.5)])
def test_alpha_shortcut_reachability(alpha, tau):
    """Every non-edge (p, z) of the alpha-CG has an out-neighbour p' of p with
    D(p', z) < D(p, z) / alpha (the shortcut-reachability argument of Sec. 3.3)."""
    n = 90
    X = _scaled_points(n, 2, 7)
    X64 = X.astype(np.float64)
    G = _alpha_cg(X, alpha, tau)
    for p in range(n):
        nb = set(G[p])
        for z in range(n):
            if z == p or z in nb:
                continue
            dz = np.linalg.norm(X64[list(nb)] - X64[z], axis=1)
            assert dz.min() < np.linalg.norm(X64[p] - X64[z]) / alpha


def test_build_invariants_random():
    X = synth.generate("gauss", 600, 8, seed=9)
    R, L, alpha, tau = 8, 24, 1.2, 0.05
    G = oracle.build_graph(X, alpha, tau, R, L)
    n = len(X)
    # phase 2 lists are exactly Alg. 2 on the exact candidate lists
    for p in range(0, n, 37):
        assert G.fwd[p, : G.fdeg[p]].tolist() == oracle.prune(X, p, G.cand[p], alpha, tau, R).tolist()
    inl = [[] for _ in range(n)]
    for u in range(n):
        for v in G.fwd[u, : G.fdeg[u]]:
            inl[v].append(u)
    for p in range(n):
        out = G.adj3[p, : G.deg3[p]].tolist()
        assert len(out) == G.deg3[p] <= R and len(set(out)) == len(out) and p not in out
        V = list(dict.fromkeys(G.fwd[p, : G.fdeg[p]].tolist() + inl[p]))
        if len(V) <= R:
            assert sorted(out) == sorted(V)  # assigned directly
        else:
            assert set(out) <= set(V)


def test_phase2_equals_alpha_cg_when_unbounded():
    X = _scaled_points(60, 2, 4)
    n = len(X)
    G = oracle.build_graph(X, 1.3, 0.2, n, n - 1)
    cg = _alpha_cg(X, 1.3, 0.2)
    for p in range(n):
        assert G.fwd[p, : G.fdeg[p]].tolist() == cg[p].tolist()


def _reachable(adj, deg, s):
    seen, stack = {s}, [s]
    while stack:
        u = stack.pop()
        for v in adj[u, : deg[u]]:
            if int(v) not in seen:
                seen.add(int(v))
                stack.append(int(v))
    return seen


def test_connectivity_repair_on_clusters():
    """Exact candidate lists on separated clusters leave the clusters disconnected; phase 4
    must make every point reachable from the entry point, adding edges only from reached
    points into unreached ones, at most R + slots per row."""
    X = synth.generate("sift", 3000, 32, seed=3)
    G = oracle.build_graph(X, 1.2, 0.0, 12, 30)
    n = len(X)
    assert len(_reachable(G.adj3, G.deg3, G.entry)) < n  # the phase-3 graph is disconnected
    assert len(_reachable(G.adj, G.deg, G.entry)) == n
    assert G.repair_edges > 0 and G.repair_rounds >= 1
    assert np.all(G.deg <= 12 + oracle.REPAIR_SLOTS)
    for p in range(n):  # phase-3 edges kept in place, repair edges appended
        assert np.array_equal(G.adj[p, : G.deg3[p]], G.adj3[p, : G.deg3[p]])
    # the first round's edges, from the searches for the unreached points on the phase-3 graph:
    # r(p) = the first result with a free slot; points without in-edges go first, each to its
    # r(p) while that row has room, else each named r takes the smallest p naming it
    reach0 = _reachable(G.adj3, G.deg3, G.entry)
    U = np.array(sorted(set(range(n)) - reach0), np.int32)
    ids, _, _, _ = oracle.search(X, G.adj3, G.deg3, G.entry, X[U], oracle.CONNECT_L,
                                 oracle.CONNECT_L)
    Rs = 12 + oracle.REPAIR_SLOTS
    has_in = np.zeros(n, bool)
    for u in range(n):
        has_in[G.adj3[u, : G.deg3[u]]] = True
    rp = {}
    for p, row in zip(U, ids):
        r = next((int(c) for c in row if c >= 0 and G.deg3[c] < Rs), None)
        if r is not None:
            rp[int(p)] = r
    taken = {}
    if any(not has_in[p] for p in rp):
        for p in sorted(rp):
            r = rp[p]
            if not has_in[p] and G.deg3[r] + len(taken.get(r, [])) < Rs:
                taken.setdefault(r, []).append(p)
    else:
        for p in sorted(rp):
            taken.setdefault(rp[p], [p])
    assert taken
    for r, ps in taken.items():
        assert r in reach0
        assert G.adj[r, G.deg3[r]: G.deg3[r] + len(ps)].tolist() == ps


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_connect_links_every_source_once(seed):
    """Phase 4 on random sparse graphs in which most points have no in-edge (every row points
    into 120 'popular' points): at the end every point is reachable from the entry, the
    phase-3 edges are in place, no point receives more than one repair edge (a linked point is
    reached and never named again), and every point without an in-edge other than the entry
    receives exactly one (nothing else can reach it)."""
    rng = np.random.default_rng(seed)
    n, d, R = 400, 8, 4
    X = rng.standard_normal((n, d)).astype(np.float32)
    adj3 = np.full((n, R), -1, np.int32)
    deg3 = np.zeros(n, np.int32)
    targets = rng.choice(n, 120, replace=False)
    for u in range(n):
        k = int(rng.integers(0, R + 1))
        vs = rng.choice(targets[targets != u], k, replace=False)
        adj3[u, :k] = vs
        deg3[u] = k
    entry = int(targets[0])
    adj, deg, added, rounds = oracle.connect(X, adj3, deg3, entry, slots=8, Lc=16)
    assert len(_reachable(adj, deg, entry)) == n and rounds >= 1
    rep_in = np.zeros(n, np.int64)
    for u in range(n):
        assert np.array_equal(adj[u, : deg3[u]], adj3[u, : deg3[u]])
        np.add.at(rep_in, adj[u, deg3[u]: deg[u]], 1)
    assert rep_in.sum() == added and rep_in.max() == 1
    has_in = np.zeros(n, bool)
    for u in range(n):
        has_in[adj3[u, : deg3[u]]] = True
    sources = [p for p in range(n) if not has_in[p] and p != entry]
    assert len(sources) > n // 2
    assert all(rep_in[p] == 1 for p in sources)


ADAPT = (0.9, 1.6, 0.05)  # the paper's setting (Sec. 4.4): alpha0, alpha_max, dalpha


def _alphas(a0, am, da):
    return [a0 + i * da for i in range(int(math.floor((am - a0) / da + 0.5)) + 1)]


def _first_alpha_set(X, p, V, R, tau=0.0):
    """Alg. 4 restated through the fixed-alpha prune: the first alpha_i whose set reaches R/2,
    else the last one tried."""
    for a in _alphas(*ADAPT):
        S = oracle.prune(X, p, V, a, tau, R)
        if 2 * len(S) >= R:
            return S
    return S


def test_adaptive_build_reduces_to_fixed():
    """alpha0 = alpha_max = alpha: Alg. 4 tries exactly one alpha, so the build equals the
    fixed-alpha build in every phase."""
    X = synth.generate("gauss", 400, 8, seed=11)
    G = oracle.build_graph(X, 1.2, 0.0, 8, 24, connect_L=0)
    H = oracle.build_graph(X, 0.0, 0.0, 8, 24, connect_L=0, adaptive=(1.2, 1.2, 0.05))
    assert np.array_equal(G.cand, H.cand) and np.array_equal(G.fwd, H.fwd)
    assert np.array_equal(G.adj, H.adj) and np.array_equal(G.deg, H.deg)


@pytest.mark.parametrize("kind,n,d,R,L", [("gauss", 500, 8, 10, 30), ("sift", 600, 16, 12, 40)])
def test_adaptive_build_phase2_and_phase3(kind, n, d, R, L):
    """Phase 2 (Alg. 3): every list is Alg. 4 on the candidate list -- the fixed-alpha prune at
    the first alpha_i reaching R/2.  Phase 3: every merged set above R is pruned the same way;
    smaller ones are kept whole in (D, id) order."""
    X = synth.generate(kind, n, d, seed=12)
    G = oracle.build_graph(X, 0.0, 0.0, R, L, connect_L=0, adaptive=ADAPT)
    used = set()
    for p in range(n):
        S = _first_alpha_set(X, p, G.cand[p], R)
        assert list(G.fwd[p][:G.fdeg[p]]) == list(S)
        assert np.all(G.fwd[p][G.fdeg[p]:] == -1)
    inl = [[] for _ in range(n)]
    for u in range(n):
        for v in G.fwd[u][:G.fdeg[u]]:
            inl[v].append(u)
    for p in range(n):
        f = list(G.fwd[p][:G.fdeg[p]])
        V = f + [u for u in inl[p] if u not in f]
        got = list(G.adj[p][:G.deg[p]])
        if len(V) <= R:
            D = ((X[V].astype(np.float64) - X[p]) ** 2).sum(1)
            assert got == [V[i] for i in np.lexsort((V, D))]
        else:
            assert got == list(_first_alpha_set(X, p, np.array(V, np.int32), R))
            used.add(p)
    assert used  # the re-prune branch was exercised


def test_tau_grid_search_in_oracle():
    """The tau grid search runs tau = 0, the coarse values 10, 1, 0.1, 0.01, 0.001, then halves
    and doubles the best; a target no graph reaches picks tau = 0 with every width exhausted;
    an easy target is reached at the first width by every graph and the fewest hops win."""
    X = synth.generate("gauss", 600, 8, seed=4)
    Q = synth.generate("gauss", 40, 8, seed=1004)
    gt, _ = oracle.knn(X, 5, rows=Q)
    Ls = [5, 8, 16]
    best, trials = oracle.tune_tau(X, 1.2, 10, 24, Q, 5, gt, Ls, 0.5)
    taus = [t["tau"] for t in trials]
    assert taus[:6] == [0.0, 10.0, 1.0, 0.1, 0.01, 0.001]
    reached = [t for t in trials if t["L"] > 0]
    assert all(t["L"] == 5 for t in reached)
    b = min(reached, key=lambda t: (t["hops_mean"], t["tau"]))
    assert best == b["tau"]
    bc = min([t for t in trials[:6] if t["L"] > 0], key=lambda t: (t["hops_mean"], t["tau"]))
    fine = set(taus[6:])
    assert fine <= ({bc["tau"] / 2, bc["tau"] * 2} if bc["tau"] > 0 else {0.0005})
    best2, trials2 = oracle.tune_tau(X, 1.2, 10, 24, Q, 5, gt, Ls, 1.01)
    assert best2 == 0.0 and all(t["L"] == 0 for t in trials2)
    # a graph's hop count at a width is Alg. 1's own: recompute one trial directly
    G = oracle.build_graph(X, 1.2, trials[2]["tau"], 10, 24)
    _, _, _, hops = oracle.search(X, G.adj, G.deg, G.entry, Q, 5, 5)
    assert trials[2]["hops_mean"] == hops.sum() / len(Q)
