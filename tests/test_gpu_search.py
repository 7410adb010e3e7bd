"""GPU parity of the batched beam search (K7) against the FP64 oracle's Alg. 1 on the same
graph: identical ids and hop counts for every query; NDC >= the oracle's (the GPU's visited
filter is lossy, recomputing a point never changes the queue)."""
import numpy as np
import pytest

import oracle
from paper_2510_05975_gb300 import synth

from gpu_util import host, lib, need_gpu, tensor

pytestmark = pytest.mark.gpu


def _search_check(X, Q, idx, cng, k, L, **kw):
    adj, deg, R, entry = cng.cng_graph(idx)
    A, D = host(adj), host(deg)
    res = cng.cng_search(idx, tensor(Q), k=k, L=L, **kw)
    ids, ds, ndc, hops = oracle.search(X, A, D, entry, Q, k, L)
    g_ids = host(res["ids"])
    bad = np.flatnonzero((g_ids != ids).any(axis=1))
    assert bad.size == 0, f"queries {bad[:10]} differ"
    assert np.array_equal(host(res["hops"]), hops)
    assert np.all(host(res["ndc"]) >= ndc)
    assert np.allclose(host(res["dists"]), ds, rtol=2e-6)
    return res


@pytest.mark.parametrize("kind,n,d,R,Lb,L,k", [
    ("gauss", 3000, 32, 16, 64, 32, 10),
    ("gauss", 3000, 32, 16, 64, 200, 10),
    ("sift", 3001, 128, 32, 128, 64, 10),
    ("deep", 2500, 96, 24, 80, 16, 1),
])
def test_search_matches_oracle(kind, n, d, R, Lb, L, k):
    need_gpu()
    cng = lib()
    X = synth.generate(kind, n, d, seed=5)
    Q = synth.generate(kind, 257, d, seed=1005, )
    idx, _ = cng.cng_build(tensor(X), alpha=1.2, R=R, L=Lb)
    _search_check(X, Q, idx, cng, k, L)
    _search_check(X, Q, idx, cng, k, L, use_graph=True)
    _search_check(X, Q, idx, cng, k, L, use_graph=True)  # replay of the cached graph
    cng.cng_free(idx)


def test_search_gauss10k_and_recall():
    need_gpu()
    cng = lib()
    w = synth.WORKLOADS["gauss10k"]
    X, Q = w.base(), w.queries()
    idx, _ = cng.cng_build(tensor(X), alpha=w.alpha, R=w.R, L=w.L)
    res = _search_check(X, Q, idx, cng, w.k, 64)
    gt, _ = oracle.knn(X, w.k, rows=Q)
    assert oracle.recall(host(res["ids"]), gt) > 0.8
    cng.cng_free(idx)


def test_search_host_buffers_and_edges():
    need_gpu()
    cng = lib()
    X = synth.generate("gauss", 1500, 16, seed=4)
    Q = synth.generate("gauss", 33, 16, seed=6)
    idx, _ = cng.cng_build(tensor(X), alpha=1.2, R=8, L=24)
    res = cng.cng_search(idx, Q, k=5, L=5)  # host in, host out
    adj, deg, R, entry = cng.cng_graph(idx)
    ids, ds, ndc, hops = oracle.search(X, host(adj), host(deg), entry, Q, 5, 5)
    assert np.array_equal(res["ids"], ids)
    # empty batch and max_hops
    r0 = cng.cng_search(idx, tensor(Q[:0]), k=5, L=8)
    assert r0["ids"].shape[0] == 0
    r1 = cng.cng_search(idx, tensor(Q), k=5, L=16, max_hops=2)
    assert np.all(host(r1["hops"]) <= 2)
    with pytest.raises(cng.CngError):
        cng.cng_search(idx, tensor(Q), k=9, L=8)
    cng.cng_free(idx)


def test_search_launch_shapes_and_autotune():
    """Queries per CTA (1 or 8 warps per block) and the autotuned shape give the oracle's ids
    and hops; the autotuned shape is reported and reused."""
    need_gpu()
    cng = lib()
    X = synth.generate("sift", 5000, 128, seed=6)
    Q = synth.generate("sift", 700, 128, seed=1006)
    idx, _ = cng.cng_build(tensor(X), alpha=1.2, R=16, L=64)
    for wpb in (1, 8):
        r = _search_check(X, Q, idx, cng, 10, 40, warps_per_block=wpb, with_stats=True)
        assert r["stats"]["warps_per_block"] == wpb
    a = _search_check(X, Q, idx, cng, 10, 40, warps_per_block=0, with_stats=True)
    b = _search_check(X, Q, idx, cng, 10, 40, warps_per_block=0, with_stats=True)
    assert a["stats"]["warps_per_block"] in (1, 2, 4, 8)
    assert a["stats"]["hash_slots"] in (512, 1024, 2048)
    assert (a["stats"]["warps_per_block"], a["stats"]["hash_slots"]) == \
        (b["stats"]["warps_per_block"], b["stats"]["hash_slots"])
    cng.cng_free(idx)


def test_search_mixed_query_exactness():
    """Integer data: integer queries inside the data's range take the exact integer path
    (8-bit rows); non-integer or out-of-range queries take the FP32 path with FP64 near-tie
    decisions.  A batch mixing both gives the oracle's ids and hops for every query."""
    need_gpu()
    cng = lib()
    X = synth.generate("sift", 4000, 128, seed=8)
    Q = synth.generate("sift", 300, 128, seed=1008)
    Q[100:200] += 0.37                      # not integers
    Q[200:250, 0] = float(X.max()) + 3.0    # outside the data's range
    idx, st = cng.cng_build(tensor(X), alpha=1.2, R=16, L=64)
    assert st["exact_int"] == 1
    _search_check(X, Q, idx, cng, 10, 32)
    _search_check(X, Q, idx, cng, 10, 32, use_graph=True)
    cng.cng_free(idx)


@pytest.fixture(scope="module")
def sift_r32():
    need_gpu()
    cng = lib()
    X = synth.generate("sift", 6000, 128, seed=21)
    Q = synth.generate("sift", 400, 128, seed=1021)
    idx, st = cng.cng_build(tensor(X), alpha=1.2, R=32, L=128)
    assert st["exact_int"] == 1
    yield cng, X, Q, idx
    cng.cng_free(idx)


@pytest.mark.parametrize("L", [12, 40, 100, 256])
def test_search_register_queue(sift_r32, L):
    """Exact 8-bit data runs on the register-queue kernel (queues of 32, 64, 128 and 256
    entries): the oracle's ids and hops for every query, through hops with more than 32 new
    points (row stride 40, merged 32 at a time) and, at L = 256, visited filters that overflow
    (their points are looked up in the queue, so NDC exceeds the oracle's)."""
    cng, X, Q, idx = sift_r32
    r = _search_check(X, Q, idx, cng, 10, L, warps_per_block=4, with_stats=True)
    _search_check(X, Q, idx, cng, 10, L, use_graph=True)
    if L == 256:
        adj, deg, R, entry = cng.cng_graph(idx)
        _, _, ndc, _ = oracle.search(X, host(adj), host(deg), entry, Q, 10, L)
        assert (host(r["ndc"]) > ndc).any()
