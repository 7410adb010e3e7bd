"""GPU parity of the learned early-stop path (not in the paper): training kernels vs the FP64
oracle's gradients and Adam, search-state features vs the oracle's traces, learned-stop
decisions vs the oracle's rule on the same BF16 weights, and a training run that learns."""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import mlp
from paper_2510_05975_gb300 import synth

from gpu_util import host, lib, need_gpu, tensor

pytestmark = pytest.mark.gpu


def test_gradient_matches_oracle():
    need_gpu()
    cng = lib()
    rng = np.random.default_rng(0)
    P = mlp.init(3)
    X = rng.standard_normal((1000, 16))
    y = (rng.random(1000) < 0.6).astype(np.float64)
    loss, g = cng.cng_mlp_grad(tensor(P.astype(np.float32)), tensor(X.astype(np.float32)),
                               tensor(y.astype(np.float32)))
    ref_loss, ref_g = mlp.loss_and_grad(P.astype(np.float32).astype(np.float64),
                                        X.astype(np.float32).astype(np.float64), y)
    assert abs(float(loss.item()) - ref_loss) <= 1e-5 * abs(ref_loss)
    err = np.abs(host(g).astype(np.float64) - ref_g)
    assert err.max() <= 1e-4 * np.abs(ref_g).max() + 1e-7


def test_adam_matches_oracle():
    need_gpu()
    cng = lib()
    rng = np.random.default_rng(1)
    P, g = rng.standard_normal(cng.CNG_STOP_NPARAMS), rng.standard_normal(cng.CNG_STOP_NPARAMS)
    m, v = rng.standard_normal(cng.CNG_STOP_NPARAMS) * 0.1, rng.random(cng.CNG_STOP_NPARAMS) * 0.1
    tp, tm, tv = (tensor(a.astype(np.float32)) for a in (P, m, v))
    cng.cng_mlp_adam(tp, tm, tv, tensor(g.astype(np.float32)), 7, 1e-3)
    rp, rm, rv = mlp.adam(P, m, v, g, 7, lr=1e-3)
    assert np.allclose(host(tp), rp, rtol=1e-5, atol=1e-6)
    assert np.allclose(host(tm), rm, rtol=1e-5, atol=1e-7)
    assert np.allclose(host(tv), rv, rtol=1e-5, atol=1e-7)


@pytest.fixture(scope="module")
def small_index():
    need_gpu()
    cng = lib()
    X = synth.generate("sift", 4000, 32, seed=11)
    Q = synth.generate("sift", 150, 32, seed=12, centre_seed=11)
    idx, _ = cng.cng_build(tensor(X), alpha=1.2, R=16, L=48)
    adj, deg, Rs, entry = cng.cng_graph(idx)
    yield cng, X, Q, idx, host(adj), host(deg), entry
    cng.cng_free(idx)


def test_trace_features_match_oracle(small_index):
    cng, X, Q, idx, A, D, entry = small_index
    T = 300
    tr = cng.cng_trace(idx, tensor(Q), 10, 24, T)
    ref = oracle.search_ex(X, A, D, entry, Q, 10, 24, max_trace=T)
    hops = host(tr["hops"])
    assert np.array_equal(hops, ref["hops"])
    assert np.array_equal(host(tr["tlc"]), ref["tlc"])
    assert np.array_equal(host(tr["ids"]), ref["ids"])
    F = host(tr["feats"]).astype(np.float64)
    for q in range(len(Q)):
        h = min(hops[q], T)
        assert np.allclose(F[q, :h], ref["feats"][q, :h], rtol=1e-4, atol=2e-5), q


@pytest.mark.parametrize("every,gate", [(2, 0), (1, 3)])
def test_learned_stop_matches_oracle_rule(small_index, every, gate):
    cng, X, Q, idx, A, D, entry = small_index
    rng = np.random.default_rng(5)
    P = mlp.init(9).astype(np.float32)
    ref = oracle.search_ex(X, A, D, entry, Q, 10, 24, max_trace=400)
    F = ref["feats"]
    flat = np.concatenate([F[q, : ref["hops"][q]] for q in range(len(Q))])
    mu, sg = flat.mean(0).astype(np.float32), (flat.std(0) + 1e-3).astype(np.float32)
    model = cng.cng_stop_import(P, mu, sg)
    _, _, _, Pb = cng.cng_stop_export(model)
    omodel = np.concatenate([Pb.astype(np.float64), mu.astype(np.float64), sg.astype(np.float64)])
    thr = 0.6
    zthr = math.log(thr / (1 - thr))
    res = cng.cng_search(idx, tensor(Q), k=10, L=24, mode=cng.CNG_SEARCH_LEARNED, model=model,
                         threshold=thr, check_every=every, min_stable=gate)
    orc = oracle.search_ex(X, A, D, entry, Q, 10, 24, model=omodel, zthr=zthr, check_every=every,
                           min_stable=gate)
    checked = 0
    for q in range(len(Q)):
        # skip queries whose decision is within 1e-3 of the threshold at some check up to the stop
        stop_at = orc["hops"][q]
        close = any(abs(oracle.mlp_logit(omodel, F[q, t - 1]) - zthr) < 1e-3
                    for t in range(every, stop_at + 1, every))
        if close:
            continue
        checked += 1
        assert host(res["hops"])[q] == orc["hops"][q], q
        assert np.array_equal(host(res["ids"])[q], orc["ids"][q]), q
        assert bool(host(res["flags"])[q] & 4) == bool(orc["stopped"][q]), q
    assert checked >= len(Q) * 0.8
    model.free()


def test_training_learns_and_stops_early(small_index):
    cng, X, Q, idx, A, D, entry = small_index
    Tq = synth.generate("sift", 1500, 32, seed=13, centre_seed=11)
    model, st = cng.cng_stop_train(idx, tensor(Tq), k=10, L=48, epochs=6, seed=3)
    assert st["samples"] > 1500 and 0 < st["positives"] < st["samples"]
    assert st["loss_last"] < st["loss_first"]
    fixed = cng.cng_search(idx, tensor(Q), k=10, L=48)
    learned = cng.cng_search(idx, tensor(Q), k=10, L=48, mode=cng.CNG_SEARCH_LEARNED, model=model,
                             threshold=0.9, check_every=1)
    gt, _ = oracle.knn(X, 10, rows=Q)
    r_f = oracle.recall(host(fixed["ids"]), gt)
    r_l = oracle.recall(host(learned["ids"]), gt)
    assert host(learned["hops"]).mean() < host(fixed["hops"]).mean()
    assert r_l >= r_f - 0.05
    model.free()
