"""Batched coloring (bgpc_color_batched): every graph of a batch gets exactly
the coloring it gets alone, which is the oracle's RS coloring of that graph."""
import numpy as np
import pytest
import torch

import graphgen as gg
import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bg():
    import paper_1701_02628_gb300 as m
    from paper_1701_02628_gb300 import build
    build.build()
    return m


@pytest.fixture(scope="module")
def ctx(bg):
    return bg.Context(0)


def mixed_batch():
    gs = [gg.random_bipartite(2000, 2000, 5, seed=1),
          gg.stencil9(40),
          gg.chung_lu(6000, 12, 700, 2.1, seed=8),
          gg.from_nets(5, []),                      # no nets at all
          gg.from_nets(1, [[0]]),
          gg.from_nets(300, [list(range(300))]),    # one clique net
          gg.random_bipartite(777, 50, 9, seed=3),
          gg.chung_lu(3000, 16, 900, 2.1, seed=5)]
    gs += [gg.batch_graph(17, i, lo=1e3, hi=2e4) for i in range(6)]
    return gs


@pytest.mark.parametrize("policy", [O.FF, O.B1, O.B2])
def test_batched_equals_single_and_oracle(bg, ctx, policy):
    graphs = mixed_batch()
    dgs = [bg.DeviceGraph.from_host(g, "cuda:0") for g in graphs]
    cols, st, rounds, ncol = bg.bgpc_color_batched(ctx, dgs, policy=policy, validate=True)
    torch.cuda.synchronize()
    max_rounds = 0
    for k, (g, dg, c) in enumerate(zip(graphs, dgs, cols)):
        ref = O.rs_color(g, policy, nthreads=8)
        got = c.cpu().numpy()
        assert np.array_equal(got, ref.colors), f"graph {k} differs"
        assert rounds[k] == ref.rounds, f"graph {k} rounds"
        assert ncol[k] == (int(ref.colors.max()) + 1 if g.n_a else 0)
        single, sst, _ = bg.bgpc_color(ctx, dg, policy=policy)
        assert np.array_equal(single.cpu().numpy(), got)
        max_rounds = max(max_rounds, ref.rounds)
    assert st["rounds"] == max_rounds
    assert st["w_per_round"][0] == sum(g.n_a for g in graphs)


def test_batched_semantic_parameters(bg, ctx):
    graphs = [gg.chung_lu(4000, 10, 500, 2.1, seed=s) for s in range(5)]
    dgs = [bg.DeviceGraph.from_host(g, "cuda:0") for g in graphs]
    for chunk, waves, big_net in [(7, 3, 4), (64, 1, O.NO_BIG), (32, 16, 0)]:
        cols, st, rounds, _ = bg.bgpc_color_batched(ctx, dgs, chunk=chunk, waves=waves,
                                                    big_net=big_net)
        for g, c, r in zip(graphs, cols, rounds):
            ref = O.rs_color(g, O.FF, chunk=chunk, waves=waves, big_net=big_net)
            assert np.array_equal(c.cpu().numpy(), ref.colors)
            assert r == ref.rounds


def test_batched_rejects_bad_arguments(bg, ctx):
    g = bg.DeviceGraph.from_host(gg.random_bipartite(100, 80, 3, seed=1), "cuda:0")
    rank = torch.arange(100, dtype=torch.int32, device="cuda:0")
    with pytest.raises(bg.BgpcError):
        bg.bgpc_color_batched(ctx, [g, g], rank=rank)
    with pytest.raises(bg.BgpcError):
        bg.bgpc_color_batched(ctx, [g], stop_after_waves=2)
    # the same graph twice is fine: the batch copies it side by side
    cols, _, _, _ = bg.bgpc_color_batched(ctx, [g, g])
    assert torch.equal(cols[0], cols[1])


def test_batch_streams_is_a_mapping_parameter(bg, ctx):
    graphs = [gg.batch_graph(5, i, lo=1e3, hi=3e4) for i in range(20)]
    dgs = [bg.DeviceGraph.from_host(g, "cuda:0") for g in graphs]
    ref = None
    for k in (1, 3, 8, 16):
        cols, st, rounds, ncol = bg.bgpc_color_batched(ctx, dgs, batch_streams=k)
        got = [c.cpu().numpy() for c in cols]
        if ref is None:
            ref = (got, rounds, ncol, st["trav_total"])
            for g, c in zip(graphs[:4], got):
                assert np.array_equal(c, O.rs_color(g).colors)
        else:
            assert all(np.array_equal(a, b) for a, b in zip(got, ref[0]))
            assert (rounds, ncol, st["trav_total"]) == ref[1:]
    with pytest.raises(bg.BgpcError):
        bg.bgpc_color_batched(ctx, dgs, batch_streams=-1)
