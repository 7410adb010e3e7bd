"""Hand-worked pins for the oracle's learned-stop trace (the 16 per-hop features, tlc, labels and
the stop rule on top of Alg. 1), its phase-4 connectivity repair (Alg. 3 phase 4), and its
whole-list soundness check of Def. 2 / Alg. 2.  The expected values come from the golden files
(worked by hand, each with its reasoning), never from the oracle itself."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import mlp


def _load(golden_dir, name):
    with open(os.path.join(golden_dir, name)) as f:
        return json.load(f)


def _value(expr: str) -> float:
    # the golden's feature expressions use only ln(integer), integers, '-' and '/'
    return float(eval(expr, {"__builtins__": {}}, {"ln": math.log}))


def _trace_graph(g):
    X = np.array([[x, 0.0] for x in g["x"]], np.float32)
    n, stride = len(X), g["stride"]
    adj = np.full((n, stride), -1, np.int32)
    deg = np.zeros(n, np.int32)
    for p, row in enumerate(g["adj"]):
        adj[p, : len(row)] = row
        deg[p] = len(row)
    return X, adj, deg


def test_trace_features_hand_worked(golden_dir):
    g = _load(golden_dir, "trace_1d.json")
    X, adj, deg = _trace_graph(g)
    q = np.zeros((1, 2), np.float32)
    T = len(g["hops"]) + 2  # room past the last hop: those rows stay untouched (NaN)
    r = oracle.search_ex(X, adj, deg, g["entry"], q, g["k"], g["L"], max_trace=T)
    fin = g["final"]
    assert r["ids"][0].tolist() == fin["ids"]
    assert r["dists"][0].tolist() == pytest.approx(fin["dists"], abs=0)
    assert (int(r["ndc"][0]), int(r["hops"][0]), int(r["tlc"][0])) == (fin["ndc"], fin["hops"], fin["tlc"])
    F = r["feats"][0]
    for h in g["hops"]:
        t = h["t"]
        want = [_value(e) for e in h["f"]]
        got = F[t - 1].tolist()
        for j in range(16):
            assert got[j] == pytest.approx(want[j], rel=1e-12, abs=1e-12), (t, j, got[j], want[j])
        # the hand-worked queue state behind the features
        Q = h["Q"]
        assert want[3] == pytest.approx(math.log(Q[min(g["k"], len(Q)) - 1][0]) - math.log(g["x"][g["entry"]]))
        assert h["U"] == sum(1 for e in Q if not e[2])
        assert g["dk_hist"][t] == Q[min(g["k"], len(Q)) - 1][0]
    assert np.all(np.isnan(F[len(g["hops"]):]))
    # label of hop t: 1 iff t >= the final tlc
    labels = [int(h["t"] >= r["tlc"][0]) for h in g["hops"]]
    assert labels == fin["labels"]


def _model(spec):
    p = np.zeros(mlp.N_PARAMS)
    H, NF = 64, 16
    off = {"W1": 0, "b1": H * NF, "W2": H * NF + H, "b2": H * NF + H + H * H,
           "w3": H * NF + 2 * H + H * H, "b3": H * NF + 3 * H + H * H}
    for name, v in spec.items():
        base = name.split("[")[0]
        idx = [int(s.rstrip("]")) for s in name.split("[")[1:]]
        if base == "W1":
            o = off["W1"] + idx[0] * NF + idx[1]
        elif base == "W2":
            o = off["W2"] + idx[0] * H + idx[1]
        elif base in ("b1", "b2", "w3"):
            o = off[base] + idx[0]
        else:
            o = off["b3"]
        p[o] = v
    assert off["b3"] == mlp.N_PARAMS - 1
    return np.concatenate([p, np.zeros(16), np.ones(16)])


def test_stop_rule_hand_worked(golden_dir):
    g = _load(golden_dir, "trace_1d.json")
    X, adj, deg = _trace_graph(g)
    q = np.zeros((1, 2), np.float32)
    for c in g["stop_cases"]:
        r = oracle.search_ex(X, adj, deg, g["entry"], q, g["k"], g["L"], model=_model(c["model"]),
                             zthr=c["zthr"], check_every=c["check_every"], min_stable=c["min_stable"])
        got = (int(r["hops"][0]), int(r["ndc"][0]), r["ids"][0].tolist(), int(r["stopped"][0]))
        assert got == (c["hops"], c["ndc"], c["ids"], c["stopped"]), c["why"]


def test_connect_hand_worked(golden_dir):
    g = _load(golden_dir, "connect_1d.json")
    for c in g["cases"]:
        X = np.array([[x, 0.0] for x in c["x"]], np.float32)
        adj3 = np.array(c["adj3"], np.int32)
        deg3 = (adj3 >= 0).sum(axis=1).astype(np.int32)
        if c["adj"] is None:
            with pytest.raises(ValueError):
                oracle.connect(X, adj3, deg3, c["entry"], slots=c["slots"], Lc=c["Lc"])
            continue
        adj, deg, added, rounds = oracle.connect(X, adj3, deg3, c["entry"], slots=c["slots"], Lc=c["Lc"])
        assert [adj[p, : deg[p]].tolist() for p in range(len(X))] == c["adj"], c["why"]
        assert (added, rounds) == (c["added"], c["rounds"]), c["why"]


def test_check_rule_on_hand_worked_lists(golden_dir):
    """Def. 2 soundness on the 2-D example: {a, b, e} (Vamana rule, alpha 1.2) is sound; adding
    g (pruned by b: 1.562 > 1.2 * 1.044) or putting e before b breaks it."""
    g = _load(golden_dir, "prune_2d.json")
    names = list(g["points"])
    X = np.array([g["p"]] + [g["points"][k] for k in names], np.float32)
    ix = {k: i + 1 for i, k in enumerate(names)}
    n = len(X)

    def rows(lst):
        L = np.full((n, 6), -1, np.int32)
        c = np.zeros(n, np.int32)
        L[0, : len(lst)] = [ix[k] for k in lst]
        c[0] = len(lst)
        return L, c

    for lst, alpha, tau, want in (
        (["a", "b", "e"], 1.2, 0.0, 0),
        (["a", "b", "e", "f"], 1.6, 0.0, 0),
        (["a", "b", "g", "e", "f"], 1.2, 0.3, 0),
        (["a", "b", "g", "e"], 1.2, 0.0, 3),   # g pruned by b
        (["a", "e", "b"], 1.2, 0.0, 2),        # out of (D, id) order
        (["a", "a"], 1.2, 0.0, 1),             # duplicate
    ):
        L, c = rows(lst)
        nb, bad = oracle.check_rule(X, L, c, alpha, tau)
        assert (nb, int(bad[0])) == (int(want != 0), want), (lst, alpha, tau)


def test_check_rule_accepts_oracle_lists_and_catches_planted_errors():
    from paper_2510_05975_gb300 import synth

    X = synth.generate("gauss", 600, 8, seed=4)
    G = oracle.build_graph(X, 1.2, 0.1, 10, 40)
    nb, _ = oracle.check_rule(X, G.fwd, G.fdeg, 1.2, 0.1)
    assert nb == 0
    # a candidate the rule pruned, appended to a kept list, is caught
    p = int(np.flatnonzero(G.fdeg < 10)[0])
    kept = set(G.fwd[p, : G.fdeg[p]].tolist())
    u = next(int(v) for v in G.cand[p] if int(v) not in kept)
    fwd = G.fwd.copy()
    fdeg = G.fdeg.copy()
    S = [int(v) for v in G.cand[p] if int(v) in kept or int(v) == u]  # (D, id) order kept
    fwd[p, : len(S)] = S
    fdeg[p] = len(S)
    nb, bad = oracle.check_rule(X, fwd, fdeg, 1.2, 0.1)
    assert nb == 1 and bad[p] == 3
