"""Pins for the learned-stop oracle (an addition to the paper's method): finite-difference
gradients, closed-form loss values, Adam's first step, C and numpy forward agreement, and the
search trace's invariants."""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_2510_05975_gb300 import synth


def test_bce_closed_forms():
    assert mlp.bce([0.0], [1.0]) == pytest.approx(math.log(2), abs=1e-15)
    assert mlp.bce([0.0], [0.0]) == pytest.approx(math.log(2), abs=1e-15)
    assert mlp.bce([50.0], [1.0]) == pytest.approx(math.exp(-50), rel=1e-6)
    assert mlp.bce([-3.0], [1.0]) == pytest.approx(3 + math.log1p(math.exp(-3)), abs=1e-15)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = mlp.init(1) * 0.5 + rng.standard_normal(mlp.N_PARAMS) * 0.01
    X = rng.standard_normal((24, 16))
    y = (rng.random(24) < 0.4).astype(np.float64)
    loss, g = mlp.loss_and_grad(p, X, y)
    idx = rng.choice(mlp.N_PARAMS, 80, replace=False)
    idx = np.concatenate([idx, [mlp.N_PARAMS - 1]])  # the output bias
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (mlp.loss_and_grad(p + e, X, y)[0] - mlp.loss_and_grad(p - e, X, y)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(g[i]), (i, fd, g[i])


def test_adam_first_step_is_lr_sign():
    p = np.zeros(5)
    g = np.array([1.0, -2.0, 0.5, 0.0, 3.0])
    p1, m, v = mlp.adam(p, np.zeros(5), np.zeros(5), g, 1, lr=0.01)
    expect = -0.01 * g / (np.abs(g) + 1e-8)
    assert np.allclose(p1, expect, atol=1e-12)


def test_c_forward_matches_numpy():
    rng = np.random.default_rng(3)
    p = mlp.init(2)
    mu, sg = rng.standard_normal(16), rng.uniform(0.5, 2, 16)
    model = np.concatenate([p, mu, sg])
    for _ in range(5):
        f = rng.standard_normal(16)
        z, _ = mlp.forward(p, ((f - mu) / sg)[None])
        assert oracle.mlp_logit(model, f) == pytest.approx(float(z[0]), rel=1e-12, abs=1e-12)


def test_trace_features_and_labels():
    X = synth.generate("gauss", 800, 8, seed=1)
    Q = synth.generate("gauss", 40, 8, seed=2)
    G = oracle.build_graph(X, 1.2, 0.0, 10, 24)
    plain = oracle.search(X, G.adj, G.deg, G.entry, Q, 5, 20)
    tr = oracle.search_ex(X, G.adj, G.deg, G.entry, Q, 5, 20, max_trace=400)
    assert np.array_equal(tr["ids"], plain[0]) and np.array_equal(tr["hops"], plain[3])
    F = tr["feats"]
    for qi in range(len(Q)):
        h = tr["hops"][qi]
        assert np.all(np.isfinite(F[qi, :h])) and np.all(np.isnan(F[qi, h:]))
        assert np.allclose(F[qi, :h, 1], np.log1p(np.arange(1, h + 1)))  # f1 = ln(1 + t)
        assert np.all(F[qi, :h, 13] >= 0) and np.all(F[qi, :h, 13] <= 1)
        assert F[qi, h - 1, 13] == 0  # every entry explored when Alg. 1 stops
        full = np.flatnonzero(np.round(F[qi, :h, 14] * 20) >= 5)  # hops with |Q| >= k
        assert np.all(np.diff(F[qi, full, 3]) <= 1e-12)  # then Dk never increases
        assert 0 <= tr["tlc"][qi] <= h


def test_learned_stop_rule_in_oracle():
    X = synth.generate("gauss", 800, 8, seed=1)
    Q = synth.generate("gauss", 30, 8, seed=3)
    G = oracle.build_graph(X, 1.2, 0.0, 10, 24)
    p = np.zeros(mlp.N_PARAMS)
    model = np.concatenate([p, np.zeros(16), np.ones(16)])
    model[mlp.N_PARAMS - 1] = 1.0  # constant logit 1
    r = oracle.search_ex(X, G.adj, G.deg, G.entry, Q, 5, 20, model=model, zthr=0.5, check_every=3)
    assert np.all(r["stopped"] == 1) and np.all(r["hops"] == 3)
    r2 = oracle.search_ex(X, G.adj, G.deg, G.entry, Q, 5, 20, model=model, zthr=1.5, check_every=3)
    assert np.all(r2["stopped"] == 0)


def test_learned_stop_gate_in_oracle():
    """min_stable: with a constant stop logit, each query stops at its first check hop t whose
    top-k ids have been unchanged for min_stable hops (t - tlc_t >= min_stable, with tlc_t from
    the plain search's features); a gate longer than any search never stops one."""
    X = synth.generate("gauss", 800, 8, seed=1)
    Q = synth.generate("gauss", 30, 8, seed=3)
    G = oracle.build_graph(X, 1.2, 0.0, 10, 24)
    model = np.concatenate([np.zeros(mlp.N_PARAMS), np.zeros(16), np.ones(16)])
    model[mlp.N_PARAMS - 1] = 1.0  # constant logit 1
    plain = oracle.search_ex(X, G.adj, G.deg, G.entry, Q, 5, 20, max_trace=400)
    for g, ce in ((2, 1), (3, 2)):
        r = oracle.search_ex(X, G.adj, G.deg, G.entry, Q, 5, 20, model=model, zthr=0.5,
                             check_every=ce, min_stable=g)
        for qi in range(len(Q)):
            h = plain["hops"][qi]
            since = np.rint(np.exp(plain["feats"][qi, :h, 12]) - 1).astype(int)  # t - tlc_t
            ok = [t for t in range(1, h + 1) if t % ce == 0 and since[t - 1] >= g]
            if ok:
                assert r["stopped"][qi] == 1 and r["hops"][qi] == ok[0], qi
            else:
                assert r["stopped"][qi] == 0 and r["hops"][qi] == h, qi
    r = oracle.search_ex(X, G.adj, G.deg, G.entry, Q, 5, 20, model=model, zthr=0.5,
                         check_every=1, min_stable=10 ** 6)
    assert np.all(r["stopped"] == 0) and np.array_equal(r["hops"], plain["hops"])
