"""FP64 CPU oracle for the alpha-CNG hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg import this
package.  The CUDA library under ``paper_2510_05975_gb300/`` never imports it and shares no
code with it.

``cng_oracle.c`` holds the graph arithmetic (canonical distance, exact candidate lists,
Def. 2 / Alg. 2 pruning, Alg. 4 adaptive pruning, Alg. 3 phase 3 reverse merge, Alg. 1
beam search); this module compiles it with gcc on first use (``-O2 -ffp-contract=off``,
OpenMP when available) and wraps it with ctypes.  ``mlp.py`` holds the FP64 learned-stop
network.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cng_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libcng_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle library (gcc, OpenMP if the compiler has it). Returns its path."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]
    tmp = _LIB + f".tmp{os.getpid()}"
    try:
        subprocess.run(base + ["-fopenmp", _SRC, "-o", tmp, "-lm"], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + [_SRC, "-o", tmp, "-lm"], check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32, i64, dbl, vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
            lib.or_sqdist.restype = dbl
            lib.or_sqdist.argtypes = [vp, vp, ctypes.c_int]
            lib.or_dist.restype = dbl
            lib.or_dist.argtypes = [vp, vp, ctypes.c_int]
            lib.or_knn.restype = ctypes.c_int
            lib.or_knn.argtypes = [vp, i64, vp, i64, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp]
            lib.or_centroid.restype = None
            lib.or_centroid.argtypes = [vp, i64, ctypes.c_int, vp]
            lib.or_entry.restype = i32
            lib.or_entry.argtypes = [vp, i64, ctypes.c_int]
            lib.or_prune.restype = ctypes.c_int
            lib.or_prune.argtypes = [vp, i64, ctypes.c_int, i64, vp, ctypes.c_int, dbl, dbl,
                                     ctypes.c_int, vp]
            lib.or_prune_adaptive.restype = ctypes.c_int
            lib.or_prune_adaptive.argtypes = [vp, i64, ctypes.c_int, i64, vp, ctypes.c_int, dbl,
                                              dbl, dbl, dbl, ctypes.c_int, vp, vp]
            lib.or_build.restype = ctypes.c_int
            lib.or_build.argtypes = [vp, i64, ctypes.c_int, dbl, dbl, ctypes.c_int, ctypes.c_int,
                                     vp, vp, vp, vp, vp, vp]
            lib.or_build_ex.restype = ctypes.c_int
            lib.or_build_ex.argtypes = [vp, i64, ctypes.c_int, dbl, dbl, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, dbl, dbl, dbl, vp, vp, vp, vp, vp, vp]
            lib.or_search.restype = ctypes.c_int
            lib.or_search.argtypes = [vp, i64, ctypes.c_int, vp, vp, ctypes.c_int, i32, vp, i64,
                                      ctypes.c_int, ctypes.c_int, vp, vp, vp, vp]
            lib.or_connect.restype = ctypes.c_int
            lib.or_connect.argtypes = [vp, i64, ctypes.c_int, vp, vp, ctypes.c_int, i32, ctypes.c_int,
                                       vp]
            lib.or_mlp_logit.restype = dbl
            lib.or_mlp_logit.argtypes = [vp, vp]
            lib.or_search_ex.restype = ctypes.c_int
            lib.or_search_ex.argtypes = [vp, i64, ctypes.c_int, vp, vp, ctypes.c_int, i32, vp, i64,
                                         ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, vp, dbl,
                                         ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, vp]
            lib.or_beam_candidates.restype = ctypes.c_int
            lib.or_beam_candidates.argtypes = [vp, i64, ctypes.c_int, vp, vp, ctypes.c_int, i32,
                                               ctypes.c_int, ctypes.c_int, vp, vp, vp]
            lib.or_build_beam.restype = ctypes.c_int
            lib.or_build_beam.argtypes = [vp, i64, ctypes.c_int, dbl, dbl, ctypes.c_int, ctypes.c_int,
                                          dbl, dbl, dbl, vp, ctypes.c_int, i32, ctypes.c_int,
                                          ctypes.c_int, vp, vp, vp, vp, vp]
            lib.or_check_rule.restype = i64
            lib.or_check_rule.argtypes = [vp, i64, ctypes.c_int, vp, vp, ctypes.c_int, dbl, dbl, vp]
            lib.or_num_threads.restype = ctypes.c_int
            lib.or_num_threads.argtypes = []
            _lib = lib
    return _lib


def _f32(x) -> np.ndarray:
    x = np.asarray(x)
    if x.dtype == np.float16:  # fp16 -> fp32 widening is exact
        x = x.astype(np.float32)
    return np.ascontiguousarray(x, dtype=np.float32)


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return int(_load().or_num_threads())


def sqdist(x, y) -> float:
    """Canonical squared distance: left-to-right FP64 sum of squared differences."""
    x, y = _f32(x).ravel(), _f32(y).ravel()
    assert x.size == y.size
    return float(_load().or_sqdist(_p(x), _p(y), x.size))


def dist(x, y) -> float:
    """Canonical distance sqrt(sqdist), IEEE double."""
    x, y = _f32(x).ravel(), _f32(y).ravel()
    assert x.size == y.size
    return float(_load().or_dist(_p(x), _p(y), x.size))


def knn(base, L: int, rows=None, exclude_self: bool | None = None):
    """Exact (D, id)-ordered L nearest points of ``base`` for each row (default: base itself,
    self excluded by id).  Returns (ids int32 [m, L], dist float64 [m, L])."""
    base = _f32(base)
    if rows is None:
        rows, ex = base, True if exclude_self is None else exclude_self
    else:
        rows, ex = _f32(rows), bool(exclude_self)
    n, d = base.shape
    m = rows.shape[0]
    ids = np.empty((m, L), np.int32)
    ds = np.empty((m, L), np.float64)
    rc = _load().or_knn(_p(base), n, _p(rows), m, d, L, int(ex), _p(ids), _p(ds))
    if rc != 0:
        raise ValueError(f"or_knn failed ({rc})")
    return ids, ds


def centroid(X) -> np.ndarray:
    X = _f32(X)
    c = np.empty(X.shape[1], np.float64)
    _load().or_centroid(_p(X), X.shape[0], X.shape[1], _p(c))
    return c


def entry(X) -> int:
    X = _f32(X)
    return int(_load().or_entry(_p(X), X.shape[0], X.shape[1]))


def prune(X, p: int, V, alpha: float, tau: float, R: int) -> np.ndarray:
    """Alg. 2 (Def. 2 rule) for point p on candidate ids V (any order), cut at R kept."""
    X = _f32(X)
    V = np.ascontiguousarray(V, dtype=np.int32)
    S = np.empty(max(R, 1), np.int32)
    ns = _load().or_prune(_p(X), X.shape[0], X.shape[1], int(p), _p(V), V.size, float(alpha),
                          float(tau), int(R), _p(S))
    if ns < 0:
        raise ValueError(f"or_prune failed ({ns})")
    return S[:ns].copy()


def prune_adaptive(X, p: int, V, alpha0: float, alpha_max: float, dalpha: float, tau: float,
                   R: int):
    """Alg. 4; returns (kept ids, alpha used)."""
    X = _f32(X)
    V = np.ascontiguousarray(V, dtype=np.int32)
    S = np.empty(max(R, 1), np.int32)
    a = ctypes.c_double(0.0)
    ns = _load().or_prune_adaptive(_p(X), X.shape[0], X.shape[1], int(p), _p(V), V.size,
                                   float(alpha0), float(alpha_max), float(dalpha), float(tau),
                                   int(R), _p(S), ctypes.byref(a))
    if ns < 0:
        raise ValueError(f"or_prune_adaptive failed ({ns})")
    return S[:ns].copy(), a.value


def check_rule(X, lists, cnt, alpha: float, tau: float):
    """Def. 2 / Alg. 2 soundness of every kept list: lists [n, stride] (row p's first cnt[p]
    entries) must be distinct valid ids != p in (D(p, .), id) order, with no member pruned by
    an earlier one.  Returns (number of unsound rows, per-row code: 0 sound, 1 bad id or
    duplicate, 2 order, 3 a pair the rule prunes)."""
    X = _f32(X)
    lists = np.ascontiguousarray(lists, np.int32)
    cnt = np.ascontiguousarray(cnt, np.int32)
    n, d = X.shape
    if lists.shape[0] != n or cnt.shape[0] != n:
        raise ValueError("lists and cnt need one row per point")
    bad = np.empty(n, np.int32)
    nb = _load().or_check_rule(_p(X), n, d, _p(lists), _p(cnt), lists.shape[1], float(alpha),
                               float(tau), _p(bad))
    if nb < 0:
        raise ValueError(f"or_check_rule failed ({nb})")
    return int(nb), bad


REPAIR_SLOTS = 8  # row slots beyond R for phase-4 connectivity edges
CONNECT_L = 32    # beam width of the phase-4 searches


class Graph:
    """Oracle construction result (Alg. 3 phases 1-4 with exact candidates).

    cand, fwd/fdeg (phase 2), adj3/deg3 (phase 3, stride R), adj/deg (final, stride
    R + REPAIR_SLOTS, after phase 4), entry, repair_edges, repair_rounds."""

    def __init__(self, entry, cand, fwd, fdeg, adj3, deg3):
        self.entry, self.cand, self.fwd, self.fdeg, self.adj3, self.deg3 = entry, cand, fwd, fdeg, adj3, deg3
        self.adj, self.deg, self.repair_edges, self.repair_rounds = adj3, deg3, 0, 0

    def out(self, p: int) -> np.ndarray:
        return self.adj[p, : self.deg[p]]


def connect(X, adj3, deg3, entry_id: int, slots: int = REPAIR_SLOTS, Lc: int = CONNECT_L):
    """Alg. 3 phase 4 on a copy: returns (adj [n, R + slots], deg, edges added, rounds)."""
    X = _f32(X)
    n, d = X.shape
    R = adj3.shape[1]
    adj = np.full((n, R + slots), -1, np.int32)
    adj[:, :R] = adj3
    deg = np.ascontiguousarray(deg3, np.int32).copy()
    rounds = ctypes.c_int32(0)
    added = _load().or_connect(_p(X), n, d, _p(adj), _p(deg), R + slots, int(entry_id), int(Lc),
                               ctypes.byref(rounds))
    if added < 0:
        raise ValueError(f"or_connect failed ({added})")
    return adj, deg, added, rounds.value


def build_graph(X, alpha: float, tau: float, R: int, L: int, connect_L: int = CONNECT_L,
                repair_slots: int = REPAIR_SLOTS, adaptive=None) -> Graph:
    """Alg. 3 with exact candidates.  adaptive = (alpha0, alpha_max, dalpha) prunes with Alg. 4
    in phases 2 and 3 (alpha is then unused); None prunes with the fixed alpha."""
    X = _f32(X)
    n, d = X.shape
    e = ctypes.c_int32(-1)
    cand = np.empty((n, L), np.int32)
    fwd = np.empty((n, R), np.int32)
    fdeg = np.empty(n, np.int32)
    adj = np.empty((n, R), np.int32)
    deg = np.empty(n, np.int32)
    a0, am, da = adaptive if adaptive is not None else (0.0, 0.0, 0.0)
    rc = _load().or_build_ex(_p(X), n, d, float(alpha), float(tau), int(R), int(L),
                             int(adaptive is not None), float(a0), float(am), float(da),
                             ctypes.byref(e), _p(cand), _p(fwd), _p(fdeg), _p(adj), _p(deg))
    if rc != 0:
        raise ValueError(f"or_build failed ({rc})")
    G = Graph(int(e.value), cand, fwd, fdeg, adj, deg)
    if connect_L > 0:
        G.adj, G.deg, G.repair_edges, G.repair_rounds = connect(X, adj, deg, G.entry, repair_slots,
                                                                connect_L)
    return G


def beam_candidates(X, adj, deg, entry_id: int, L: int, C: int):
    """Alg. 3 phase 2 candidates (Sec. 4.1): for each point p, Alg. 1 on the graph (adj, deg)
    from entry_id with queue size L and x_p as the query; of every point whose distance was
    computed, the C closest by (D, id) with p excluded.  Returns (ids [n, C] padded with -1,
    dists [n, C] float64 padded with inf, counts [n])."""
    X = _f32(X)
    adj = np.ascontiguousarray(adj, dtype=np.int32)
    deg = np.ascontiguousarray(deg, dtype=np.int32)
    n, d = X.shape
    ids = np.empty((n, C), np.int32)
    ds = np.empty((n, C), np.float64)
    cnt = np.empty(n, np.int32)
    rc = _load().or_beam_candidates(_p(X), n, d, _p(adj), _p(deg), adj.shape[1], int(entry_id),
                                    int(L), int(C), _p(ids), _p(ds), _p(cnt))
    if rc != 0:
        raise ValueError(f"or_beam_candidates failed ({rc})")
    return ids, ds, cnt


def build_graph_beam(X, alpha: float, tau: float, R: int, C: int, K: int, Lb: int,
                     connect_L: int = CONNECT_L, repair_slots: int = REPAIR_SLOTS,
                     adaptive=None, knn_graph=None) -> Graph:
    """Alg. 3 with the paper's candidate route: G0 = a K-NN graph (knn_graph [n, K], default the
    exact one), the navigating node of the exact route (the point nearest the centroid; the
    paper finds it by a beam search on G0), candidates = beam_candidates(G0, queue Lb, C), then
    phases 2-4 as build_graph.  Graph.cand holds the [n, C] candidate lists."""
    X = _f32(X)
    n, d = X.shape
    G0 = knn(X, K)[0] if knn_graph is None else np.ascontiguousarray(knn_graph, np.int32)
    e = entry(X)
    cand = np.empty((n, C), np.int32)
    fwd = np.empty((n, R), np.int32)
    fdeg = np.empty(n, np.int32)
    adj = np.empty((n, R), np.int32)
    deg = np.empty(n, np.int32)
    a0, am, da = adaptive if adaptive is not None else (0.0, 0.0, 0.0)
    rc = _load().or_build_beam(_p(X), n, d, float(alpha), float(tau), int(R),
                               int(adaptive is not None), float(a0), float(am), float(da),
                               _p(G0), int(G0.shape[1]), int(e), int(Lb), int(C), _p(cand),
                               _p(fwd), _p(fdeg), _p(adj), _p(deg))
    if rc != 0:
        raise ValueError(f"or_build_beam failed ({rc})")
    G = Graph(int(e), cand, fwd, fdeg, adj, deg)
    if connect_L > 0:
        G.adj, G.deg, G.repair_edges, G.repair_rounds = connect(X, adj, deg, G.entry, repair_slots,
                                                                connect_L)
    return G


def search(X, adj, deg, entry_id: int, Q, k: int, L: int):
    """Alg. 1 for every query. Returns (ids [nq,k], dist [nq,k] float64, ndc [nq], hops [nq])."""
    X, Q = _f32(X), _f32(Q)
    adj = np.ascontiguousarray(adj, dtype=np.int32)
    deg = np.ascontiguousarray(deg, dtype=np.int32)
    n, d = X.shape
    nq = Q.shape[0]
    ids = np.empty((nq, k), np.int32)
    ds = np.empty((nq, k), np.float64)
    ndc = np.empty(nq, np.int32)
    hops = np.empty(nq, np.int32)
    rc = _load().or_search(_p(X), n, d, _p(adj), _p(deg), adj.shape[1], int(entry_id), _p(Q), nq,
                           int(k), int(L), _p(ids), _p(ds), _p(ndc), _p(hops))
    if rc != 0:
        raise ValueError(f"or_search failed ({rc})")
    return ids, ds, ndc, hops


NF = 16


def search_ex(X, adj, deg, entry_id: int, Q, k: int, L: int, max_trace: int = 0, model=None,
              zthr: float = 0.0, check_every: int = 1, min_stable: int = 0):
    """Alg. 1 with per-hop search-state features (learned early stop) and, if ``model`` (the
    parameter vector followed by mu[16], sigma[16]) is given, the learned stop rule: the model
    is consulted after hops t with t % check_every == 0 whose top-k ids have not changed for
    min_stable hops.
    Returns dict(ids, dists, ndc, hops, tlc, stopped, feats [nq, max_trace, 16] or None)."""
    X, Q = _f32(X), _f32(Q)
    adj = np.ascontiguousarray(adj, dtype=np.int32)
    deg = np.ascontiguousarray(deg, dtype=np.int32)
    n, d = X.shape
    nq = Q.shape[0]
    out = dict(ids=np.empty((nq, k), np.int32), dists=np.empty((nq, k), np.float64),
               ndc=np.empty(nq, np.int32), hops=np.empty(nq, np.int32), tlc=np.empty(nq, np.int32),
               stopped=np.empty(nq, np.int32),
               feats=np.full((nq, max_trace, NF), np.nan) if max_trace else None)
    mdl = None if model is None else np.ascontiguousarray(model, np.float64)
    rc = _load().or_search_ex(_p(X), n, d, _p(adj), _p(deg), adj.shape[1], int(entry_id), _p(Q), nq,
                              int(k), int(L), int(max_trace),
                              _p(out["feats"]) if max_trace else None, _p(out["tlc"]),
                              None if mdl is None else _p(mdl), float(zthr), int(check_every), int(min_stable),
                              _p(out["ids"]), _p(out["dists"]), _p(out["ndc"]), _p(out["hops"]),
                              _p(out["stopped"]))
    if rc != 0:
        raise ValueError(f"or_search_ex failed ({rc})")
    return out


def mlp_logit(model, f) -> float:
    mdl = np.ascontiguousarray(model, np.float64)
    f = np.ascontiguousarray(f, np.float64)
    return float(_load().or_mlp_logit(_p(mdl), _p(f)))


def recall(found_ids, true_ids) -> float:
    """Recall@k = |KNN(q) & Res(q)| / k averaged over queries (Sec. 5.1, Metrics)."""
    found_ids = np.asarray(found_ids)
    true_ids = np.asarray(true_ids)
    k = true_ids.shape[1]
    hit = sum(len(set(a.tolist()) & set(b.tolist())) for a, b in zip(found_ids, true_ids))
    return hit / (k * true_ids.shape[0])


def mips_augment(X):
    """Rows for maximum-inner-product search as Euclidean search (the library's CNG_IP metric;
    the paper builds its graph over a metric space, Sec. 2.1, and has no inner-product variant):
    x' = [x, sqrt(M^2 - |x|^2)] with |x|^2 summed in FP64 over the coordinates in order (each
    square is exact), M^2 = max |x|^2, and the correctly rounded FP64 root rounded to FP32.
    Returns (X' float32 [n, d + 1], M^2)."""
    X = _f32(X)
    sq = X.astype(np.float64) ** 2
    nrm2 = np.cumsum(sq, axis=1)[:, -1]  # sequential left-to-right sums
    M2 = float(nrm2.max())
    extra = np.sqrt(M2 - nrm2).astype(np.float32)
    return np.concatenate([X, extra[:, None]], axis=1), M2


def mips_queries(Q):
    """Queries for an augmented index: q' = [q, 0], so |q' - x'|^2 = |q|^2 + M^2 - 2 <q, x>."""
    Q = _f32(Q)
    return np.concatenate([Q, np.zeros((Q.shape[0], 1), np.float32)], axis=1)


def tune_tau(X, alpha: float, R: int, L: int, Q, k: int, gt_ids, search_Ls, target: float):
    """The grid search of tau on held-out queries (Sec. 4.4, parameter configuration): tau = 0, then
    the coarse values 10, 1, 0.1, 0.01, 0.001, then t / 2 and 2 t around the best coarse value t
    (0.0005 when t = 0).  A trial's score is the smallest width in search_Ls whose mean
    Recall@k reaches `target` and the mean hops there (the recall summed query by query in
    order).  Best: reaches the target, then fewest mean hops, then smaller tau.
    Returns (best_tau, trials as dicts in the order run)."""
    gt = [set(int(v) for v in row) for row in np.asarray(gt_ids)]
    done = []

    def run(tau):
        if any(t["tau"] == tau for t in done):
            return
        G = build_graph(X, alpha, tau, R, L)
        tr = dict(tau=tau, L=0, recall=0.0, hops_mean=0.0)
        for Ls in search_Ls:
            ids, _, _, hops = search(X, G.adj, G.deg, G.entry, Q, k, int(Ls))
            rec = 0.0
            for q in range(len(Q)):
                rec += sum(1 for v in ids[q] if int(v) in gt[q]) / k
            tr["recall"] = rec / len(Q)
            tr["hops_mean"] = float(int(hops.astype(np.int64).sum())) / len(Q)
            if tr["recall"] >= target:
                tr["L"] = int(Ls)
                break
        done.append(tr)

    def key(t):
        return (0 if t["L"] > 0 else 1, t["hops_mean"] if t["L"] > 0 else 0.0, t["tau"])

    for tau in (0.0, 10.0, 1.0, 0.1, 0.01, 0.001):
        run(tau)
    best = min(done, key=key)
    for tau in ((best["tau"] / 2, best["tau"] * 2) if best["tau"] > 0 else (0.0005, 0.0005)):
        run(tau)
    best = min(done, key=key)
    return (best["tau"] if best["L"] > 0 else 0.0), done
