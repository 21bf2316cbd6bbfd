"""GPU parity of the learned-order calls against the float64 oracle
(oracle/order.py): features, bfloat16 weights, MLP forward, gradient, Adam,
rank from scores, and the learned rank fed to the coloring.

Tolerances.  u = 2^-24 is the float32 unit roundoff.  A float32 sum of k
terms computed in any order differs from the exact sum by at most
(k-1) u (sum of |terms|) to first order; the GPU evaluates every dot product
and every reduction in float32 with at most K terms, so each output is held
to |gpu - oracle| <= K u A, where A is the same expression evaluated on the
absolute values of every term (computed below in float64).  Integer results
(ranks, the bfloat16 bit patterns) are compared exactly."""
import math

import numpy as np
import pytest
import torch

import graphgen as gg
import oracle as O
from oracle import order as OO

pytestmark = pytest.mark.gpu
U = 2.0 ** -24


@pytest.fixture(scope="module")
def bg():
    import paper_1701_02628_gb300 as m
    from paper_1701_02628_gb300 import build
    build.build()
    return m


@pytest.fixture(scope="module")
def ctx(bg):
    return bg.Context(0)


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to("cuda:0", dtype).contiguous()


def init_params(seed):
    return gg.mlp_init(seed)


@pytest.mark.parametrize("name", ["rb", "cl", "edge"])
def test_features(bg, ctx, name):
    g = {"rb": lambda: gg.random_bipartite(2000, 1500, 7, seed=4),
         "cl": lambda: gg.chung_lu(5000, 12, 900, 2.1, seed=9),
         "edge": lambda: gg.from_nets(6, [[0, 1, 2], [0, 2], [4], [0, 1, 2, 4]])}[name]()
    T = 3 if name == "edge" else 64
    X = bg.features(ctx, bg.DeviceGraph.from_host(g, "cuda:0"), big_net=T).cpu().numpy()
    ref = OO.features(g, T)
    # float(log1p) of the same double statistics: within one float32 rounding
    # plus the double log1p error, i.e. 2 ulp of float32
    assert np.all(np.abs(X - ref) <= 2 * np.spacing(np.abs(ref).astype(np.float32)) + 1e-30)


def test_bf16_weights(bg, ctx):
    rng = np.random.default_rng(3)
    w = (rng.standard_normal(bg.MLP_PARAMS) * 10.0 ** rng.integers(-5, 4, bg.MLP_PARAMS))
    w = w.astype(np.float32)
    w[:4] = [1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), 0.0]  # ties to even
    mlp = bg.MLP(ctx, dev(w))
    got = mlp.bf16_values().cpu().numpy()
    assert np.array_equal(got.view(np.uint32), OO.bf16(w).view(np.uint32))


def forward_bound(p, X):
    """Float64 forward on absolute values: the magnitude A of every score."""
    W1, b1, W2, b2, W3, b3 = [np.abs(a) for a in OO.unpack(p)]
    a1 = np.abs(X) @ W1.T + b1
    a2 = a1 @ W2.T + b2
    return a2 @ W3 + b3, a1, a2


def test_forward(bg, ctx):
    rng = np.random.default_rng(8)
    n = 3001
    X = rng.random((n, 8)).astype(np.float32) * 4
    mlp = bg.MLP(ctx, dev(init_params(1)))
    p = mlp.bf16_values().cpu().numpy().astype(np.float64)
    s = bg.mlp_forward(ctx, mlp, dev(X)).cpu().numpy()
    ref, _ = OO.forward(p, X)
    A, _, _ = forward_bound(p, X)
    assert np.all(np.abs(s - ref) <= (8 + 64 + 64 + 3) * U * A)


def grad_bound(p, X, y):
    """Float64 backpropagation on absolute values: for every parameter, the
    sum of |terms| that its float32 gradient adds up."""
    W1, b1, W2, b2, W3, b3 = OO.unpack(p)
    s, (z1, h1, z2, h2) = OO.forward(p, X)
    n = X.shape[0]
    A, a1, a2 = forward_bound(p, X)
    ads = 2.0 * (np.abs(s - y) + (8 + 64 + 64 + 3) * U * A) / n
    m2, m1 = (z2 > 0), (z1 > 0)
    g = np.zeros(OO.N_PARAMS)
    g[OO.OFF_W3:OO.OFF_B3] = ads @ a2
    g[OO.OFF_B3] = ads.sum()
    adz2 = np.outer(ads, np.abs(W3)) * m2
    g[OO.OFF_W2:OO.OFF_B2] = (adz2.T @ a1).ravel()
    g[OO.OFF_B2:OO.OFF_W3] = adz2.sum(axis=0)
    adz1 = (adz2 @ np.abs(W2)) * m1
    g[OO.OFF_W1:OO.OFF_B1] = (adz1.T @ np.abs(X)).ravel()
    g[OO.OFF_B1:OO.OFF_W2] = adz1.sum(axis=0)
    return g


def clear_of_kinks(p, X):
    """Rows whose pre-activations are all far (relative to their float32
    error) from 0, so that both sides take the same ReLU branches."""
    _, (z1, _, z2, _) = OO.forward(p, X)
    _, a1, a2 = forward_bound(p, X)
    ok1 = np.all(np.abs(z1) > 1e3 * U * (1 + a1), axis=1)
    ok2 = np.all(np.abs(z2) > 1e3 * U * (1 + a2), axis=1)
    return ok1 & ok2


@pytest.mark.parametrize("n", [1, 255, 4099])
def test_grad(bg, ctx, n):
    rng = np.random.default_rng(n)
    mlp = bg.MLP(ctx, dev(init_params(2)))
    p = mlp.bf16_values().cpu().numpy().astype(np.float64)
    X = (rng.random((4 * n + 64, 8)) * 3).astype(np.float32)
    X = X[clear_of_kinks(p, X)][:n]
    assert X.shape[0] == n
    y = rng.random(n).astype(np.float32)
    gt, L = bg.mlp_grad(ctx, mlp, dev(X), dev(y))
    g = gt.cpu().numpy().astype(np.float64)
    ref, Lref = OO.grad(p, X, y)
    bound = grad_bound(p, X, y.astype(np.float64))
    K = n + 8 + 64 + 64 + 8
    assert np.all(np.abs(g - ref) <= K * U * bound + 1e-30)
    s, _ = OO.forward(p, X)
    ds = (8 + 64 + 64 + 3) * U * forward_bound(p, X)[0]
    r = np.abs(s - y)
    assert abs(L - Lref) <= np.mean(2 * r * ds + ds * ds) + (n + 2) * U * np.mean((r + ds) ** 2)
    g2, L2 = bg.mlp_grad(ctx, mlp, dev(X), dev(y))
    assert torch.equal(g2, gt) and L2 == L  # deterministic reduction


def test_adam_and_train_step(bg, ctx):
    rng = np.random.default_rng(4)
    w0 = init_params(3)
    mlp = bg.MLP(ctx, dev(w0))
    w, m, v = w0.astype(np.float64), np.zeros(bg.MLP_PARAMS), np.zeros(bg.MLP_PARAMS)
    am, av = np.zeros(bg.MLP_PARAMS), np.zeros(bg.MLP_PARAMS)  # magnitudes of m, v terms
    lr = 3e-3
    for t in range(1, 4):
        g = (rng.standard_normal(bg.MLP_PARAMS) * 10.0 ** rng.integers(-4, 2)).astype(np.float32)
        bg.mlp_adam(ctx, mlp, dev(g), lr)
        w, m, v = OO.adam(w, m, v, g.astype(np.float64), t, lr)
        am = 0.9 * am + 0.1 * np.abs(g)
        av = 0.999 * av + 0.001 * g.astype(np.float64) ** 2
        assert mlp.step == t
    wg = mlp.w.cpu().numpy()
    # per step: the float32 update lr * m_hat / (sqrt(v_hat) + eps) carries a
    # relative error of a few u on a ratio below 10, and w is rounded once;
    # m and v carry relative errors of a few u
    assert np.all(np.abs(wg - w) <= 3 * (lr * 10 * 16 * U + 2 * U * np.abs(w)))
    # each moment update is two products and a sum in float32 (3 roundings per
    # step, plus the rounding of the float32 constants 0.9, 0.1, 0.999, 0.001)
    assert np.all(np.abs(mlp.adam_m.cpu().numpy() - m) <= 3 * 6 * U * am)
    assert np.all(np.abs(mlp.adam_v.cpu().numpy() - v) <= 3 * 6 * U * av)
    assert np.array_equal(mlp.bf16_values().cpu().numpy().view(np.uint32),
                          OO.bf16(wg).view(np.uint32))
    # train_step == grad then adam, bit for bit
    X = (rng.random((700, 8)) * 2).astype(np.float32)
    y = rng.random(700).astype(np.float32)
    a = bg.MLP(ctx, dev(w0))
    b = bg.MLP(ctx, dev(w0))
    for _ in range(3):
        La = bg.mlp_train_step(ctx, a, dev(X), dev(y), lr)
        gb, Lb = bg.mlp_grad(ctx, b, dev(X), dev(y))
        bg.mlp_adam(ctx, b, gb, lr)
        assert La == Lb
    assert torch.equal(a.w, b.w) and torch.equal(a.w_bf16, b.w_bf16) and a.step == b.step == 3


def test_training_reduces_the_loss(bg, ctx):
    rng = np.random.default_rng(6)
    X = (rng.random((4000, 8)) * 3).astype(np.float32)
    y = (np.sin(X[:, 0]) + 0.3 * X[:, 3]).astype(np.float32)
    mlp = bg.MLP(ctx, dev(init_params(4)))
    losses = [bg.mlp_train_step(ctx, mlp, dev(X), dev(y), 3e-3) for _ in range(200)]
    assert losses[-1] < 0.2 * losses[0]


@pytest.mark.parametrize("n", [1, 255, 256, 257, 70001])
def test_rank_from_scores(bg, ctx, n):
    rng = np.random.default_rng(n)
    s = (rng.integers(-40, 40, n) / 8).astype(np.float32)  # many ties
    s[rng.random(n) < 0.05] = -0.0
    s[rng.random(n) < 0.01] = np.float32(np.inf)
    r = bg.rank_from_scores(ctx, dev(s)).cpu().numpy()
    assert np.array_equal(r, OO.rank_from_scores(s))


def test_rank_rejects_nan(bg, ctx):
    s = np.ones(300, np.float32)
    s[17] = math.nan
    with pytest.raises(bg.BgpcError):
        bg.rank_from_scores(ctx, dev(s))


def test_learned_rank_colors_validly(bg, ctx):
    g = gg.chung_lu(6000, 12, 700, 2.1, seed=8)
    dg = bg.DeviceGraph.from_host(g, "cuda:0")
    mlp = bg.MLP(ctx, dev(init_params(5)))
    rank = bg.learned_rank(ctx, dg, mlp)
    assert np.array_equal(np.sort(rank.cpu().numpy()), np.arange(g.n_a))
    colors, st, rc = bg.bgpc_color(ctx, dg, rank=rank)
    assert rc == bg.BGPC_OK and bg.bgpc_validate(ctx, dg, colors) == 0


@pytest.mark.slow
def test_fullsize_rank_and_sampled_features(bg, ctx):
    g = gg.chung_lu(1 << 22, 16.0, 50000.0, 2.1, seed=2)
    dg = bg.DeviceGraph.from_host(g, "cuda:0")
    X = bg.features(ctx, dg).cpu().numpy()
    rng = np.random.default_rng(1)
    pick = np.concatenate([[0, 1, g.n_a - 1], rng.choice(g.n_a, 3000, replace=False)])
    ref = OO.features_of(g, pick, 64)
    got = X[pick]
    assert np.all(np.abs(got - ref) <= 2 * np.spacing(np.abs(ref).astype(np.float32)) + 1e-30)
    s = (rng.integers(-1000, 1000, g.n_a) / 16).astype(np.float32)
    r = bg.rank_from_scores(ctx, dev(s)).cpu().numpy()
    assert np.array_equal(r, OO.rank_from_scores(s))


def test_learned_order_gains_over_id_order(bg, ctx):
    """What the trained order gains: the model is trained on 12 seeded graphs
    of the batched workload (targets: each vertex's first-fit color in id
    order), then colors 24 held-out graphs of the same generator (another
    seed).  The learned order uses fewer colors than id order on most of
    them, more on few, and fewer on average; every coloring stays valid and
    equals the oracle's coloring in that order."""
    dev = "cuda:0"
    train = [bg.DeviceGraph.from_host(gg.batch_graph(23, i, lo=1e3, hi=3e4), dev)
             for i in range(12)]
    mlp, losses = bg.train_order(ctx, train, torch.from_numpy(gg.mlp_init(7)).to(dev),
                                 steps=300, lr=3e-3)
    assert losses[-1] < 0.5 * losses[0]
    fewer = more = 0
    tot_id = tot_l = 0
    for i in range(24):
        g = gg.batch_graph(31, i, lo=1e3, hi=3e4)
        dg = bg.DeviceGraph.from_host(g, dev)
        _, st_id, _ = bg.bgpc_color(ctx, dg)
        rank = bg.learned_rank(ctx, dg, mlp)
        col, st_l, _ = bg.bgpc_color(ctx, dg, rank=rank)
        assert bg.bgpc_validate(ctx, dg, col) == 0
        if i < 4:  # the learned order is an ordinary rank: the oracle agrees
            ref = O.rs_color(g, rank=rank.cpu().numpy(), nthreads=8)
            assert np.array_equal(col.cpu().numpy(), ref.colors)
        fewer += st_l["colors"] < st_id["colors"]
        more += st_l["colors"] > st_id["colors"]
        tot_id += st_id["colors"]
        tot_l += st_l["colors"]
    assert fewer >= 16 and more <= 3, (fewer, more)
    assert tot_l < tot_id


def test_smallest_last_rank(bg, ctx):
    """The library's smallest-last order is the oracle's (same definition,
    separate code), and the GPU coloring in that order is the oracle's RS
    coloring in that rank; the pair cap is enforced."""
    dev = "cuda:0"
    graphs = [gg.from_nets(4, [[0, 1], [0, 2], [0, 3]]), gg.random_bipartite(800, 500, 4, seed=3),
              gg.stencil9(24), gg.chung_lu(3000, 10, 400, 2.1, seed=6),
              gg.batch_graph(29, 0, lo=1e3, hi=3e3), gg.from_nets(6, [[0, 1], [], [3, 4]])]
    for g in graphs:
        dg = bg.DeviceGraph.from_host(g, dev)
        rank, deg = bg.sl_rank(ctx, dg)
        ref, rdeg = O.sl_rank(g)
        assert np.array_equal(rank.cpu().numpy(), ref) and deg == rdeg
        col, st, _ = bg.bgpc_color(ctx, dg, rank=rank)
        rs = O.rs_color(g, rank=ref, nthreads=8)
        assert np.array_equal(col.cpu().numpy(), rs.colors)
    dg = bg.DeviceGraph.from_host(gg.random_bipartite(800, 500, 4, seed=3), dev)
    with pytest.raises(bg.BgpcError) as e:
        bg.sl_rank(ctx, dg, max_pairs=100)
    assert e.value.status == bg.BGPC_ENOMEM
