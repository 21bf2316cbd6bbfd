"""Pins of the learned-order oracle (oracle/order.py) against closed forms,
independent formulations and finite differences (no GPU)."""
import math
import struct

import numpy as np
import pytest

import graphgen as gg
from oracle import order as OO


def test_features_closed_form():
    # vertex 0 in nets of sizes 2 and 3; vertex 1 in the size-3 net only;
    # vertex 3 in no net at all
    g = gg.from_nets(4, [[0, 1, 2], [0, 2]])
    X = OO.features(g, big_net=2)
    raw0 = [2, 2.5, 3, 5, 3, 2, 1, (4 + 9) / 5]
    assert np.allclose(X[0], np.log1p(raw0), rtol=0, atol=1e-15)
    raw1 = [1, 3, 3, 3, 2, 3, 1, 3]
    assert np.allclose(X[1], np.log1p(raw1), rtol=0, atol=1e-15)
    assert np.all(X[3] == 0)


def _bf16_by_search(x: float) -> float:
    """Nearest bfloat16 to the float32 x (ties to the even mantissa), found by
    comparing the two neighbours in exact float64 arithmetic."""
    u = struct.unpack("<I", struct.pack("<f", x))[0]
    lo = u & 0xFFFF0000
    hi = lo + 0x10000
    f = lambda b: struct.unpack("<f", struct.pack("<I", b))[0]
    dlo, dhi = abs(f(lo) - x), abs(f(hi) - x)
    if dlo < dhi:
        return f(lo)
    if dhi < dlo:
        return f(hi)
    return f(lo) if ((lo >> 16) & 1) == 0 else f(hi)


def test_bf16_rounding():
    one = np.float32(1.0)
    assert OO.bf16(np.array([1.0], np.float32))[0] == one
    # exactly halfway cases round to the even mantissa
    assert OO.bf16(np.array([1 + 2 ** -8], np.float32))[0] == one
    assert OO.bf16(np.array([1 + 3 * 2 ** -8], np.float32))[0] == np.float32(1 + 2 ** -6)
    assert OO.bf16(np.array([-(1 + 3 * 2 ** -8)], np.float32))[0] == np.float32(-(1 + 2 ** -6))
    rng = np.random.default_rng(5)
    x = (rng.standard_normal(4000) * 10.0 ** rng.integers(-6, 6, 4000)).astype(np.float32)
    got = OO.bf16(x)
    want = np.array([_bf16_by_search(float(v)) for v in x], np.float32)
    assert np.array_equal(got, want)


def _rand_params(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return OO.bf16((rng.standard_normal(OO.N_PARAMS) * scale).astype(np.float32)).astype(np.float64)


def test_forward_closed_forms():
    p = np.zeros(OO.N_PARAMS)
    p[OO.OFF_B3] = 0.75
    X = np.random.default_rng(1).random((6, 8))
    s, _ = OO.forward(p, X)
    assert np.all(s == 0.75)
    # one path: h1_0 = relu(2 x_3 - 1), h2_5 = relu(3 h1_0 + 0.5), s = -2 h2_5 + 1
    p = np.zeros(OO.N_PARAMS)
    p[OO.OFF_W1 + 0 * 8 + 3] = 2.0
    p[OO.OFF_B1 + 0] = -1.0
    p[OO.OFF_W2 + 5 * 64 + 0] = 3.0
    p[OO.OFF_B2 + 5] = 0.5
    p[OO.OFF_W3 + 5] = -2.0
    p[OO.OFF_B3] = 1.0
    X = np.zeros((3, 8))
    X[:, 3] = [0.0, 0.75, 2.0]
    s, _ = OO.forward(p, X)
    h1 = np.maximum(2 * X[:, 3] - 1, 0)
    assert np.allclose(s, -2 * np.maximum(3 * h1 + 0.5, 0) + 1, rtol=0, atol=1e-15)


def test_grad_matches_finite_differences():
    rng = np.random.default_rng(11)
    p = _rand_params(3)
    X = rng.random((7, 8)) * 3
    y = rng.random(7)
    g, L = OO.grad(p, X, y)
    assert L == pytest.approx(OO.loss(p, X, y), rel=1e-14)
    # stay away from ReLU kinks so that central differences are smooth
    _, (z1, _, z2, _) = OO.forward(p, X)
    assert np.abs(z1).min() > 1e-4 and np.abs(z2).min() > 1e-4
    h = 1e-7
    idx = np.concatenate([rng.choice(OO.N_PARAMS, 300, replace=False),
                          [OO.OFF_B3, OO.OFF_W3, OO.OFF_B2, OO.OFF_B1, OO.OFF_W1]])
    for i in idx:
        e = np.zeros(OO.N_PARAMS)
        e[i] = h
        fd = (OO.loss(p + e, X, y) - OO.loss(p - e, X, y)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), i


def test_adam_closed_forms():
    rng = np.random.default_rng(2)
    w = rng.standard_normal(50)
    g = rng.standard_normal(50)
    lr = 1e-2
    # first step: m_hat = g, v_hat = g^2
    w1, m1, v1 = OO.adam(w, np.zeros(50), np.zeros(50), g, 1, lr)
    assert np.allclose(w1, w - lr * g / (np.abs(g) + OO.EPS), rtol=0, atol=1e-15)
    assert np.allclose(m1, 0.1 * g) and np.allclose(v1, 0.001 * g * g)
    # a constant gradient keeps m_hat = g and v_hat = g^2 at every step
    wt, m, v = w, np.zeros(50), np.zeros(50)
    for t in range(1, 30):
        wn, m, v = OO.adam(wt, m, v, g, t, lr)
        assert np.allclose(wn - wt, -lr * g / (np.abs(g) + OO.EPS), rtol=1e-12, atol=1e-15)
        wt = wn


def test_rank_from_scores_matches_sorted():
    rng = np.random.default_rng(7)
    for n in (1, 2, 17, 500):
        s = rng.integers(-5, 6, n).astype(np.float32) / 4  # many ties
        s[rng.random(n) < 0.1] = -0.0
        r = OO.rank_from_scores(s)
        order = sorted(range(n), key=lambda i: (-float(s[i]), i))
        want = np.empty(n, np.int32)
        want[order] = np.arange(n)
        assert np.array_equal(r, want)
        assert np.array_equal(np.sort(r), np.arange(n))
    with pytest.raises(ValueError):
        OO.rank_from_scores(np.array([1.0, math.nan], np.float32))
