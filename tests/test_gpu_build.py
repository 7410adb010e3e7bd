"""GPU parity of the build path (K0 prep, K3 entry, K1 screen, K2 rerank, K4 prune, K5/K6 merge)
against the FP64 oracle: candidate lists, phase-2 lists and the final graph must be identical
element by element (every FP32 near-tie is re-decided in FP64 on the GPU)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2510_05975_gb300 import synth

from gpu_util import host, lib, need_gpu, tensor

pytestmark = pytest.mark.gpu


def _check_graph(X, G, idx, cng, R, L):
    cand, cdist, fwd, fdeg = cng.cng_lists(idx)
    adj, deg, R_, entry = cng.cng_graph(idx)
    assert entry == G.entry
    c = host(cand)
    bad = np.flatnonzero((c != G.cand).any(axis=1))
    assert bad.size == 0, f"candidate lists differ at rows {bad[:10]}"
    fd = host(fdeg)
    assert np.array_equal(fd, G.fdeg)
    assert np.array_equal(host(fwd), G.fwd)
    assert np.array_equal(host(deg), G.deg)
    assert np.array_equal(host(adj), G.adj)
    # FP32 candidate distances within FP32 error of the canonical ones
    _, ds = oracle.knn(X, L)
    assert np.allclose(host(cdist), ds, rtol=2e-6, atol=0)


@pytest.mark.parametrize("kind,n,d,alpha,tau,R,L,screen", [
    ("gauss", 3000, 32, 1.2, 0.0, 16, 64, 0),
    ("gauss", 2777, 20, 1.3, 0.25, 12, 40, 0),
    ("sift", 3001, 128, 1.2, 0.0, 32, 128, 0),
    ("deep", 2500, 96, 1.3, 0.0, 24, 80, 0),
    ("gauss", 3000, 32, 1.2, 0.0, 16, 64, 1),
    ("sift", 3001, 128, 1.2, 0.0, 32, 128, 1),
    ("gauss", 3000, 32, 1.2, 0.0, 16, 64, 2),   # BF16 operands
    ("sift", 3001, 128, 1.2, 0.0, 32, 128, 2),
    ("gist", 2000, 960, 1.2, 0.0, 32, 128, 0),  # the GIST-like width: staged prune and merge
    ("gist", 2000, 960, 1.2, 0.0, 32, 128, 1),
    ("gist", 1003, 960, 1.2, 0.05, 16, 100, 1),  # ragged tiles, tau > 0
])
def test_build_matches_oracle(kind, n, d, alpha, tau, R, L, screen):
    need_gpu()
    cng = lib()
    X = synth.generate(kind, n, d, seed=5)
    idx, st = cng.cng_build(tensor(X), alpha=alpha, R=R, L=L, tau=tau, screen=screen, keep_lists=True)
    G = oracle.build_graph(X, alpha, tau, R, L)
    _check_graph(X, G, idx, cng, R, L)
    if kind == "sift":
        assert st["exact_int"] == 1
    assert st["screen_used"] == screen
    cng.cng_free(idx)


def test_gauss10k_full_size():
    """The 10,000 x 32 N(0,1) workload at its stated parameters (alpha 1.2, R 32, L 64)."""
    need_gpu()
    cng = lib()
    w = synth.WORKLOADS["gauss10k"]
    X = w.base()
    idx, st = cng.cng_build(tensor(X), alpha=w.alpha, R=w.R, L=w.L, keep_lists=True)
    G = oracle.build_graph(X, w.alpha, 0.0, w.R, w.L)
    _check_graph(X, G, idx, cng, w.R, w.L)
    cng.cng_free(idx)


def test_host_points_and_fp16():
    need_gpu()
    cng = lib()
    X = synth.generate("bigann16", 2000, 64, seed=3, dtype="float16")  # FP16 storage
    idx, st = cng.cng_build(X, alpha=1.2, R=16, L=48, keep_lists=True)  # host array
    G = oracle.build_graph(X.astype(np.float32), 1.2, 0.0, 16, 48)
    _check_graph(X.astype(np.float32), G, idx, cng, 16, 48)
    cng.cng_free(idx)


def test_duplicates_and_tiny_n():
    need_gpu()
    cng = lib()
    rng = np.random.default_rng(1)
    base = rng.integers(0, 4, size=(40, 3)).astype(np.float32)  # many exact duplicates and ties
    X = np.concatenate([base, base[:10]])
    n = len(X)
    idx, st = cng.cng_build(tensor(X), alpha=1.1, R=6, L=n - 1, keep_lists=True)
    G = oracle.build_graph(X, 1.1, 0.0, 6, n - 1)
    _check_graph(X, G, idx, cng, 6, n - 1)
    cng.cng_free(idx)


def test_ip_metric_requires_unit_norm():
    need_gpu()
    cng = lib()
    X = synth.generate("gauss", 500, 16, seed=2)
    with pytest.raises(cng.CngError) as e:
        cng.cng_build(tensor(X), alpha=1.2, R=8, L=16, metric=cng.CNG_IP_AS_L2)
    assert e.value.code == cng.CNG_E_INVAL
    Xu = synth.generate("deep", 500, 16, seed=2)
    idx, _ = cng.cng_build(tensor(Xu), alpha=1.3, R=8, L=16, metric=cng.CNG_IP_AS_L2)
    cng.cng_free(idx)


@pytest.mark.parametrize("kind,d,screen", [("gauss", 48, 0), ("gauss", 48, 1), ("gist", 960, 1),
                                           ("gist", 330, 1)])
def test_knn_rows_vs_oracle(kind, d, screen):
    need_gpu()
    cng = lib()
    X = synth.generate(kind, 5003, d, seed=8)
    Q = synth.generate(kind, 300, d, seed=9)
    ids, ds, st = cng.cng_knn(tensor(X), 100, rows=tensor(Q), screen=screen)
    ref, rd = oracle.knn(X, 100, rows=Q)
    assert st["screen_used"] == screen
    assert np.array_equal(host(ids), ref)
    assert np.allclose(host(ds), rd, rtol=2e-6)


def test_knn_screen_heavy_ties():
    """Lattice points (coordinates 0..3 in 8 dimensions): squared distances take fewer than 80
    values, so the screen's row buffers hold runs of equal keys far longer than the thinning
    slack between tiles.  The selection then keeps ties in buffer order, and the rerank's
    certification (with exact rescans) must still give the exact (distance, id) lists."""
    need_gpu()
    cng = lib()
    rng = np.random.default_rng(17)
    X = rng.integers(0, 4, size=(6000, 8)).astype(np.float32)
    ids, ds, st = cng.cng_knn(tensor(X), 100, screen=cng.CNG_SCREEN_TC)
    ref, rd = oracle.knn(X, 100)
    assert st["screen_used"] == 1
    assert np.array_equal(host(ids), ref)
    assert np.allclose(host(ds), rd, rtol=2e-7, atol=0)  # exact D^2, one FP32 square root


@pytest.mark.parametrize("kind,n,d,R,L", [
    ("sift", 60_001, 128, 32, 128),   # two waves of 152 row blocks and a ragged tail
    ("deep", 41_000, 96, 24, 80),
])
def test_locality_order_same_lists(kind, n, d, R, L):
    """The tensor-core screen's locality order changes speed only: candidate lists, distances,
    phase-2 lists and the final graph equal those of the input-order sweep."""
    need_gpu()
    cng = lib()
    X = tensor(synth.generate(kind, n, d, seed=9))
    out = []
    for input_order in (False, True):
        idx, st = cng.cng_build(X, alpha=1.2, R=R, L=L, keep_lists=True, input_order=input_order)
        assert st["screen_used"] == 1
        assert (st["ms_order"] > 0) != input_order
        cand, cdist, fwd, fdeg = cng.cng_lists(idx)
        adj, deg, _, entry = cng.cng_graph(idx)
        out.append([host(a) for a in (cand, cdist, fwd, fdeg, adj, deg)] + [entry])
        cng.cng_free(idx)
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("kind,n,d,R,L,screen", [
    ("gauss", 3000, 32, 16, 64, 1),    # FP32 register-resident sweep
    ("sift", 3001, 128, 32, 128, 1),   # 8-bit integer sweep
    ("deep", 2500, 96, 24, 80, 1),     # FP32 register-resident sweep, d = 96
    ("gist", 1500, 200, 16, 48, 0),    # staged sweep (rows too wide for registers)
    ("gist", 2000, 960, 32, 128, 0),   # the GIST-like width, FP32 screen
    ("gist", 2000, 960, 32, 128, 1),   # the GIST-like width, tensor-core screen
])
def test_adaptive_build_matches_oracle(kind, n, d, R, L, screen):
    """Adaptive pruning (Alg. 4 with the paper's alpha0 0.9, dalpha 0.05, alpha_max 1.6) in
    phases 2 and 3: lists and graph identical to the oracle's adaptive build."""
    need_gpu()
    cng = lib()
    grid = (0.9, 1.6, 0.05)
    X = synth.generate(kind, n, d, seed=7)
    idx, st = cng.cng_build(tensor(X), alpha=1.2, R=R, L=L, screen=screen, keep_lists=True,
                            adaptive=grid)
    G = oracle.build_graph(X, 1.2, 0.0, R, L, adaptive=grid)
    _check_graph(X, G, idx, cng, R, L)
    assert 0.9 <= st["alpha_mean"] <= 1.6
    cng.cng_free(idx)


@pytest.mark.parametrize("screen", [0, 1])
def test_mips_metric_matches_oracle(screen):
    """CNG_IP: the graph equals the oracle's graph of the augmented rows, searches with plain
    d-dimensional queries equal the oracle's Alg. 1 on the augmented queries, and the results
    are the largest inner products."""
    need_gpu()
    cng = lib()
    rng = np.random.default_rng(7)
    X = (synth.generate("gauss", 2500, 24, seed=7) * rng.uniform(0.3, 2.5, (2500, 1))).astype(np.float32)
    Q = synth.generate("gauss", 200, 24, seed=1007)
    Xa, M2 = oracle.mips_augment(X)
    idx, st = cng.cng_build(tensor(X), alpha=1.2, R=16, L=64, screen=screen, keep_lists=True,
                            metric=cng.CNG_IP)
    G = oracle.build_graph(Xa, 1.2, 0.0, 16, 64)
    _check_graph(Xa, G, idx, cng, 16, 64)
    adj, deg, _, entry = cng.cng_graph(idx)
    res = cng.cng_search(idx, tensor(Q), k=10, L=64)
    ids, ds, _, hops = oracle.search(Xa, host(adj), host(deg), entry, oracle.mips_queries(Q), 10, 64)
    assert np.array_equal(host(res["ids"]), ids)
    assert np.array_equal(host(res["hops"]), hops)
    top = np.argsort(-(Q.astype(np.float64) @ X.astype(np.float64).T), axis=1, kind="stable")[:, :10]
    assert oracle.recall(host(res["ids"]), top) > 0.9
    cng.cng_free(idx)


def test_tau_grid_search_matches_oracle():
    """cng_tune_tau runs the same trials as the oracle's grid search (graphs, widths, recalls
    and hop counts are exact) and picks the same tau."""
    need_gpu()
    cng = lib()
    X = synth.generate("gauss", 1500, 16, seed=12)
    Q = synth.generate("gauss", 120, 16, seed=1012)
    gt, _ = oracle.knn(X, 10, rows=Q)
    Ls = [10, 12, 16, 24, 32, 48]
    best, trials = cng.cng_tune_tau(tensor(X), 1.2, 16, 48, tensor(Q), 10, gt, Ls, 0.95)
    obest, otrials = oracle.tune_tau(X, 1.2, 16, 48, Q, 10, gt, Ls, 0.95)
    key = lambda ts: [(t["tau"], t["L"], t["recall"], t["hops_mean"]) for t in ts]
    assert key(trials) == key(otrials)
    assert best == obest


@pytest.mark.parametrize("kind,n,d,R,C,K,Lb,screen", [
    ("gauss", 3000, 32, 16, 48, 64, 49, 1),
    ("sift", 3001, 128, 32, 96, 128, 128, 1),   # integer data: the 8-bit exact search path
    ("gauss", 4000, 24, 16, 100, 200, 160, 0),  # G0 rows wider than 96 entries (read in slices)
    ("deep", 2500, 96, 24, 80, 96, 81, 1),
])
def test_beam_candidates_match_oracle(kind, n, d, R, C, K, Lb, screen):
    """The paper's candidate route (Alg. 3 phase 2, Sec. 4.1): candidates are the C closest
    points visited by a beam search for p on the exact K-NN graph G0; candidate lists, phase-2
    lists and the final graph equal the oracle's."""
    need_gpu()
    cng = lib()
    X = synth.generate(kind, n, d, seed=11)
    idx, st = cng.cng_build(tensor(X), alpha=1.2, R=R, L=C, screen=screen, keep_lists=True,
                            candidates=cng.CNG_CAND_BEAM, knn_K=K, beam_L=Lb)
    G = oracle.build_graph_beam(X, 1.2, 0.0, R, C, K, Lb)
    cand, _, fwd, fdeg = cng.cng_lists(idx)
    adj, deg, _, entry = cng.cng_graph(idx)
    assert entry == G.entry
    bad = np.flatnonzero((host(cand) != G.cand).any(axis=1))
    assert bad.size == 0, f"candidate lists differ at rows {bad[:10]}"
    assert np.array_equal(host(fdeg), G.fdeg) and np.array_equal(host(fwd), G.fwd)
    assert np.array_equal(host(deg), G.deg) and np.array_equal(host(adj), G.adj)
    assert st["ms_cand_search"] > 0
    cng.cng_free(idx)


def test_beam_candidates_on_a_given_approximate_graph():
    """G0 supplied by the caller (the paper builds an approximate K-NN graph): the exact 48-NN
    lists with their last 16 entries replaced by random other points; the build equals the
    oracle's route on the same G0.  A G0 with a self edge is rejected before any search."""
    need_gpu()
    cng = lib()
    X = synth.generate("gauss", 2500, 16, seed=12)
    n, K = len(X), 48
    G0, _ = oracle.knn(X, K)
    rng = np.random.default_rng(3)
    for p in range(n):
        keep = set(G0[p, :32].tolist()) | {p}
        extra = [v for v in rng.permutation(n)[:64].tolist() if v not in keep][:16]
        G0[p, 32:] = extra
    idx, _ = cng.cng_build(tensor(X), alpha=1.2, R=16, L=40, keep_lists=True,
                           candidates=cng.CNG_CAND_BEAM, beam_L=41,
                           knn_graph=torch.from_numpy(G0).cuda())
    G = oracle.build_graph_beam(X, 1.2, 0.0, 16, 40, K, 41, knn_graph=G0)
    cand, _, fwd, _ = cng.cng_lists(idx)
    adj, deg, _, _ = cng.cng_graph(idx)
    assert np.array_equal(host(cand), G.cand) and np.array_equal(host(fwd), G.fwd)
    assert np.array_equal(host(adj), G.adj) and np.array_equal(host(deg), G.deg)
    cng.cng_free(idx)
    bad = G0.copy()
    bad[7, 3] = 7
    with pytest.raises(cng.CngError) as e:
        cng.cng_build(tensor(X), alpha=1.2, R=16, L=40, candidates=cng.CNG_CAND_BEAM,
                      knn_graph=torch.from_numpy(bad).cuda())
    assert e.value.code == cng.CNG_E_INVAL


@pytest.mark.parametrize("M", [600, 2500])
def test_long_near_tie_run_in_merge(M):
    """A hub whose merged set is one long run of near-tied distances: M points on a sphere of
    radius 1 (+- 2e-7) around point 0 in 32 dimensions all keep point 0 (their nearest point),
    so its merged set holds M entries whose FP32 distances cannot order them; the GPU re-sorts
    the whole run by the canonical FP64 distance (M = 2500 exceeds the shared-memory merge and
    takes the global-scratch pass) and the graph equals the oracle's."""
    need_gpu()
    cng = lib()
    rng = np.random.default_rng(5)
    v = rng.standard_normal((M, 32))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    v *= 1.0 + 2e-7 * rng.standard_normal((M, 1))
    X = np.concatenate([np.zeros((1, 32)), v]).astype(np.float32)
    idx, st = cng.cng_build(tensor(X), alpha=1.2, R=16, L=48, keep_lists=True)
    G = oracle.build_graph(X, 1.2, 0.0, 16, 48)
    assert int((G.fwd == 0).sum()) == M  # every sphere point keeps the hub
    _check_graph(X, G, idx, cng, 16, 48)
    assert st["order_ties"] > 0
    cng.cng_free(idx)


@pytest.mark.parametrize("M", [1200, 5000])
def test_merge_prefix_of_a_large_set(M):
    """A hub whose merged set (well over 512 entries; over 2,048 for M = 5000) fills R early:
    half of M points on a sphere around point 0 at distinct radii 1 .. 1.25, the other half at
    radius 1.3 (+- 2e-7), one long near-tie run at the end of the hub's order.  Nothing is pruned
    around the hub, so Alg. 2 keeps its first R entries; the GPU orders and prunes a prefix of
    the set, never re-sorting the tail run, and the graph equals the oracle's."""
    need_gpu()
    cng = lib()
    rng = np.random.default_rng(7)
    v = rng.standard_normal((M, 32))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    h = M // 2
    r = np.concatenate([1.0 + 0.25 * np.arange(h) / h, 1.3 * (1.0 + 2e-7 * rng.standard_normal(M - h))])
    X = np.concatenate([np.zeros((1, 32)), v * r[:, None]]).astype(np.float32)
    idx, st = cng.cng_build(tensor(X), alpha=1.2, R=16, L=48, keep_lists=True)
    G = oracle.build_graph(X, 1.2, 0.0, 16, 48)
    assert int((G.fwd == 0).sum()) > 512 and G.deg[0] == 16
    _check_graph(X, G, idx, cng, 16, 48)
    cng.cng_free(idx)


def test_merge_prefix_runs_out():
    """A hub with 1,196 in-edges from 30 tight clusters (40 points each around a random
    direction, radius 1 .. 1.1): in the hub's sweep the first point of each cluster prunes the
    rest of it, so only 30 < R = 32 are kept and Alg. 2 reads the whole set; the GPU's prefix
    runs out, it orders the rest and prunes the set again, and the graph equals the oracle's."""
    need_gpu()
    cng = lib()
    rng = np.random.default_rng(9)
    u = rng.standard_normal((30, 32))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    pts = [np.zeros((1, 32))]
    for k in range(30):
        dirs = u[k] + 0.01 * rng.standard_normal((40, 32))
        dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
        pts.append(dirs * rng.uniform(1.0, 1.1, (40, 1)))
    X = np.concatenate(pts).astype(np.float32)
    idx, st = cng.cng_build(tensor(X), alpha=1.2, R=32, L=64, keep_lists=True)
    G = oracle.build_graph(X, 1.2, 0.0, 32, 64)
    assert int((G.fwd == 0).sum()) > 512 and G.deg[0] == 30
    _check_graph(X, G, idx, cng, 32, 64)
    cng.cng_free(idx)


@pytest.mark.parametrize("slots", [2, 24])
def test_repair_slots(slots):
    """Phase 4 with a given number of repair slots per row (row stride R + slots): separated
    clusters need repair edges; the final graph equals the oracle's with the same slots."""
    need_gpu()
    cng = lib()
    rng = np.random.default_rng(9)
    centres = rng.standard_normal((12, 16)) * 40.0
    X = (centres[rng.integers(0, 12, 1500)] + rng.standard_normal((1500, 16))).astype(np.float32)
    idx, st = cng.cng_build(tensor(X), alpha=1.2, R=12, L=40, keep_lists=True, repair_slots=slots)
    G = oracle.build_graph(X, 1.2, 0.0, 12, 40, repair_slots=slots)
    assert st["repair_edges"] == G.repair_edges > 0
    adj, deg, Rs, _ = cng.cng_graph(idx)
    assert Rs == 12 + slots
    assert np.array_equal(host(adj), G.adj) and np.array_equal(host(deg), G.deg)
    cng.cng_free(idx)


def test_screen_variants_give_identical_lists():
    """Every pipeline variant of the tensor-core screen (operand stages, row-buffer capacity,
    checkpoint lag) yields the same candidate lists, phase-2 lists and graph; the stats report
    the shape used."""
    need_gpu()
    cng = lib()
    X = tensor(synth.generate("sift", 40_001, 128, seed=13))
    ref = None
    shapes = set()
    for v in range(1, 7):
        idx, st = cng.cng_build(X, alpha=1.2, R=32, L=128, keep_lists=True, screen_variant=v)
        assert st["screen_variant"] == v - 1 and st["screen_stages"] >= 2
        shapes.add((st["screen_stages"], st["screen_cap"], st["screen_sync"]))
        cand, _, fwd, _ = cng.cng_lists(idx)
        adj, deg, _, _ = cng.cng_graph(idx)
        got = [host(a) for a in (cand, fwd, adj, deg)]
        cng.cng_free(idx)
        if ref is None:
            ref = got
        else:
            for a, b in zip(ref, got):
                assert np.array_equal(a, b), v
    assert len(shapes) == 6


def test_screen_autotuner_picks_a_variant():
    """At 400k points the first build of the shape times the variants on a row sample and uses
    the fastest; the lists equal those of a forced variant."""
    need_gpu()
    cng = lib()
    X = tensor(synth.generate("sift", 400_000, 128, seed=14))
    idx, st = cng.cng_build(X, alpha=1.2, R=32, L=128, keep_lists=True)
    assert 0 <= st["screen_variant"] < 6 and st["screen_cap"] >= 288
    cand_a = host(cng.cng_lists(idx)[0])
    cng.cng_free(idx)
    idx, st2 = cng.cng_build(X, alpha=1.2, R=32, L=128, keep_lists=True, screen_variant=1)
    assert np.array_equal(cand_a, host(cng.cng_lists(idx)[0]))
    cng.cng_free(idx)


def _int_clusters(n, d, seed, k=20):
    """Integer coordinates in 0..255 around k integer centres (8-bit rows, exact distances)."""
    rng = np.random.default_rng(seed)
    c = rng.integers(64, 192, (k, d))
    X = c[rng.integers(0, k, n)] + np.rint(rng.normal(0.0, 20.0, (n, d)))
    return np.clip(X, 0, 255).astype(np.float32)


@pytest.mark.parametrize("d,n,R,L,alpha,tau,seed", [
    (20, 2500, 16, 64, 1.2, 0.0, 1),     # 8-bit rows of 8 words: K = 32
    (64, 2500, 24, 100, 1.2, 0.3, 2),    # 16 words, tau > 0, list length not a multiple of 32
    (96, 2000, 32, 128, 1.3, 0.0, 3),    # 24 words: K = 96 (a partial second K atom)
    (128, 3001, 64, 128, 1.2, 0.0, 4),   # 32 words, R = 64
    (128, 2000, 32, 37, 1.0, 0.0, 5),    # a short ragged list, alpha = 1
])
def test_gram_prune_matches_oracle(d, n, R, L, alpha, tau, seed):
    """Integer data through the tensor-core Gram-tile prune and merge (phase 2b and phase 3):
    lists and graph identical to the oracle's."""
    need_gpu()
    cng = lib()
    X = _int_clusters(n, d, seed)
    idx, st = cng.cng_build(tensor(X), alpha=alpha, R=R, L=L, tau=tau, keep_lists=True)
    assert st["prune_path"] == 2
    G = oracle.build_graph(X, alpha, tau, R, L)
    _check_graph(X, G, idx, cng, R, L)
    cng.cng_free(idx)


def test_gram_prune_lattice_ties():
    """Lattice points (coordinates 0..2 in 24 dimensions, 100 of them duplicated) with alpha = 1:
    many pairs fall exactly on the rule's boundary D(p,v) = D(u,v) and duplicates sit at
    D(p,v) = 0, so the Gram tile's near-tie masks are exercised; the FP64 re-decisions give the
    oracle's lists and graph."""
    need_gpu()
    cng = lib()
    rng = np.random.default_rng(11)
    X = rng.integers(0, 3, (1400, 24))
    X = np.concatenate([X, X[:100]]).astype(np.float32)
    idx, st = cng.cng_build(tensor(X), alpha=1.0, R=12, L=48, keep_lists=True)
    assert st["prune_path"] == 2
    G = oracle.build_graph(X, 1.0, 0.0, 12, 48)
    _check_graph(X, G, idx, cng, 12, 48)
    assert st["rule_ties"] > 0
    cng.cng_free(idx)


def test_gram_merge_with_a_hub():
    """A hub with 700 near points keeps them all in its merged set (beyond the Gram tile's 128
    and the 256-entry pass), beside ordinary nodes of the Gram pass: graph equals the oracle's."""
    need_gpu()
    cng = lib()
    rng = np.random.default_rng(12)
    d = 32
    hub = np.full((1, d), 128)
    near = 128 + rng.integers(-3, 4, (700, d))
    far = rng.integers(0, 256, (800, d))
    X = np.concatenate([hub, near, far]).astype(np.float32)
    idx, st = cng.cng_build(tensor(X), alpha=1.2, R=16, L=64, keep_lists=True)
    assert st["prune_path"] == 2
    G = oracle.build_graph(X, 1.2, 0.0, 16, 64)
    assert st["merge_max_list"] > 256
    _check_graph(X, G, idx, cng, 16, 64)
    cng.cng_free(idx)


@pytest.mark.parametrize("d,n,R,L,tau,seed", [
    (128, 3001, 32, 128, 0.0, 21),   # K = 128, full tile
    (64, 2500, 24, 100, 0.3, 22),    # K = 64, tau > 0, list length not a multiple of 32
    (128, 1000, 64, 64, 0.0, 23),    # short lists, R = 64
])
def test_gram_prune_fp16_matches_oracle(d, n, R, L, tau, seed):
    """FP16 storage through the Gram-tile prune (FP32 accumulation, certified decision windows;
    pairs inside them decided again by the FP32 difference form, then FP64): lists and graph
    identical to the oracle's."""
    need_gpu()
    cng = lib()
    X = synth.generate("bigann16", n, d, seed=seed, dtype="float16")
    assert X.dtype == np.float16
    idx, st = cng.cng_build(tensor(X), alpha=1.2, R=R, L=L, tau=tau, keep_lists=True)
    assert st["prune_path"] == 3
    Xf = X.astype(np.float32)
    G = oracle.build_graph(Xf, 1.2, tau, R, L)
    _check_graph(Xf, G, idx, cng, R, L)
    cng.cng_free(idx)


def test_gram_prune_fp16_ties():
    """Half-integer lattice points in FP16 (0, 0.5, 1, 1.5 in 64 dimensions; 100 duplicated) with
    alpha = 1: exact rule boundaries and D(p,v) = 0 entries go through the open-pair path (FP32
    difference form, then FP64) and give the oracle's lists."""
    need_gpu()
    cng = lib()
    rng = np.random.default_rng(24)
    X = rng.integers(0, 4, (1400, 64)) * 0.5
    X = np.concatenate([X, X[:100]]).astype(np.float16)
    idx, st = cng.cng_build(tensor(X), alpha=1.0, R=12, L=48, keep_lists=True)
    assert st["prune_path"] == 3
    Xf = X.astype(np.float32)
    G = oracle.build_graph(Xf, 1.0, 0.0, 12, 48)
    _check_graph(Xf, G, idx, cng, 12, 48)
    assert st["rule_ties"] > 0
    cng.cng_free(idx)


@pytest.mark.parametrize("kind,d,n,R,L,alpha,tau,seed", [
    ("deep", 96, 3000, 48, 160, 1.3, 0.0, 31),    # the DEEP-like shape: lists of 160
    ("gauss", 32, 3000, 48, 250, 1.2, 0.0, 32),   # eight 32-entry chunks, ragged
    ("gauss", 20, 2500, 16, 64, 1.2, 0.25, 33),   # tau > 0, rows narrower than a chunk
    ("gist", 960, 1500, 32, 128, 1.2, 0.0, 34),   # rows of 30 chunks
])
def test_pairs_prune_matches_oracle(kind, d, n, R, L, alpha, tau, seed):
    """Float rows through the CUDA-core all-pairs prune (Gram blocks with certified windows, open
    pairs decided again by the FP32 difference form, then FP64): lists and graph identical to the
    oracle's."""
    need_gpu()
    cng = lib()
    X = synth.generate(kind, n, d, seed=seed)
    idx, st = cng.cng_build(tensor(X), alpha=alpha, R=R, L=L, tau=tau, keep_lists=True)
    assert st["prune_path"] == 4
    G = oracle.build_graph(X, alpha, tau, R, L)
    _check_graph(X, G, idx, cng, R, L)
    cng.cng_free(idx)


def test_pairs_prune_ties():
    """Half-integer lattice points in FP32 (0 .. 1.5 in 40 dimensions, 100 duplicated), alpha = 1:
    exact rule boundaries and D(p,v) = 0 entries take the open-pair path; lists equal the
    oracle's."""
    need_gpu()
    cng = lib()
    rng = np.random.default_rng(35)
    X = rng.integers(0, 4, (1400, 40)) * 0.5
    X = np.concatenate([X, X[:100]]).astype(np.float32)
    idx, st = cng.cng_build(tensor(X), alpha=1.0, R=12, L=48, keep_lists=True)
    assert st["prune_path"] == 4
    G = oracle.build_graph(X, 1.0, 0.0, 12, 48)
    _check_graph(X, G, idx, cng, 12, 48)
    assert st["rule_ties"] > 0
    cng.cng_free(idx)


def test_pairs_prune_fp16_wide_rows():
    """FP16 storage with rows wider than the FP16 Gram tile (d = 200, dpad = 256) takes the
    all-pairs path with converted FP16 loads; the merge re-prunes its sets the same way."""
    need_gpu()
    cng = lib()
    X = synth.generate("bigann16", 2000, 200, seed=36, dtype="float16")
    idx, st = cng.cng_build(tensor(X), alpha=1.2, R=24, L=96, keep_lists=True)
    assert st["prune_path"] == 4
    Xf = X.astype(np.float32)
    G = oracle.build_graph(Xf, 1.2, 0.0, 24, 96)
    _check_graph(Xf, G, idx, cng, 24, 96)
    assert st["merge_repruned"] > 0
    cng.cng_free(idx)
