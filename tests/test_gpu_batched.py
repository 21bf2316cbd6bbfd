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
        cols, st, rounds, ncol = bg.bgpc_color_batched(ctx, dgs, batch_streams=k,
                                                       batch_engine=bg.BGPC_BATCH_STREAMS)
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


# ------------------------------------------------ persistent engine mappings

def check_against_oracle(graphs, cols, rounds, ncol, policy=O.FF, **kw):
    for k, (g, c) in enumerate(zip(graphs, cols)):
        ref = O.rs_color(g, policy, nthreads=8, **kw)
        assert np.array_equal(c.cpu().numpy(), ref.colors), f"graph {k} differs"
        assert rounds[k] == ref.rounds, f"graph {k} rounds"
        assert ncol[k] == (int(ref.colors.max()) + 1 if g.n_a else 0)


@pytest.mark.parametrize("policy", [O.FF, O.B2X])
def test_persistent_every_mapping(bg, ctx, policy):
    """Every candidate of the autotuner (window width, CTAs per SM, wave-task
    span) gives the oracle's colors: the mapping never changes a result."""
    graphs = mixed_batch()
    dgs = [bg.DeviceGraph.from_host(g, "cuda:0") for g in graphs]
    first = None
    for mp in range(1, bg.BGPC_BATCH_MAPPINGS + 1):
        cols, st, rounds, ncol = bg.bgpc_color_batched(ctx, dgs, policy=policy,
                                                       batch_mapping=mp)
        got = [c.cpu().numpy() for c in cols]
        if first is None:
            check_against_oracle(graphs, cols, rounds, ncol, policy)
            first = (got, rounds, ncol, st["trav_total"], st["w_per_round"])
        else:
            assert all(np.array_equal(a, b) for a, b in zip(got, first[0])), f"mapping {mp}"
            assert (rounds, ncol, st["trav_total"], st["w_per_round"]) == first[1:]


def test_persistent_window_fallback(bg, ctx):
    """A graph whose colors outgrow the shared-memory window (a clique net of
    3000 members needs colors up to 2999) is finished by the single-graph
    engine; its neighbours in the batch are not affected."""
    graphs = [gg.from_nets(3000, [list(range(3000))]), gg.random_bipartite(900, 700, 4, seed=2),
              gg.chung_lu(20000, 16, 1500, 2.1, seed=4)]
    dgs = [bg.DeviceGraph.from_host(g, "cuda:0") for g in graphs]
    for policy in (O.FF, O.B1):
        for mp in (1, 3, 5):  # windows of 1024, 512 and 2048 colors
            cols, st, rounds, ncol = bg.bgpc_color_batched(ctx, dgs, policy=policy,
                                                           batch_mapping=mp)
            check_against_oracle(graphs, cols, rounds, ncol, policy)
            assert st["pieces_total"] >= 1  # graphs handed back to the single-graph engine


def test_persistent_replay_and_autotune(bg, ctx):
    """The first call on a batch autotunes and captures the launch in a CUDA
    graph; later calls replay it.  The replay reads the graphs' current
    contents: new graphs of the same sizes at the same addresses are colored
    correctly."""
    graphs = [gg.random_bipartite(3000, 2000, 6, seed=s) for s in (1, 2, 3)]
    dgs = [bg.DeviceGraph.from_host(g, "cuda:0") for g in graphs]
    outs = [torch.empty(g.n_a, dtype=torch.int32, device="cuda:0") for g in graphs]
    for _ in range(3):
        cols, st, rounds, ncol = bg.bgpc_color_batched(ctx, dgs, outs)
        check_against_oracle(graphs, cols, rounds, ncol)
    new = [gg.random_bipartite(3000, 2000, 6, seed=s) for s in (11, 12, 13)]
    for dg, g in zip(dgs, new):
        for dst, src in ((dg.a_ptr, g.a_ptr), (dg.a_idx, g.a_idx), (dg.b_ptr, g.b_ptr),
                         (dg.b_idx, g.b_idx)):
            dst.copy_(torch.as_tensor(src, device="cuda:0"))
    cols, st, rounds, ncol = bg.bgpc_color_batched(ctx, dgs, outs)
    check_against_oracle(new, cols, rounds, ncol)


def test_persistent_errors(bg, ctx):
    clique = bg.DeviceGraph.from_host(gg.from_nets(40, [list(range(40))]), "cuda:0")
    other = bg.DeviceGraph.from_host(gg.random_bipartite(200, 100, 3, seed=1), "cuda:0")
    with pytest.raises(bg.BgpcError) as e:
        bg.bgpc_color_batched(ctx, [other, clique], chunk=1, waves=1, big_net=bg.NO_BIG,
                              max_rounds=5)
    assert e.value.status == bg.BGPC_EROUNDS
    for kw in (dict(batch_mapping=-1), dict(batch_mapping=bg.BGPC_BATCH_MAPPINGS + 1),
               dict(batch_engine=2), dict(net_rounds=1)):
        with pytest.raises(bg.BgpcError) as e:
            bg.bgpc_color_batched(ctx, [other], **kw)
        assert e.value.status == bg.BGPC_EINVAL
    # all-empty batch
    empty = bg.DeviceGraph.from_host(gg.from_nets(0, []), "cuda:0")
    cols, st, rounds, ncol = bg.bgpc_color_batched(ctx, [empty, empty])
    assert rounds == [0, 0] and ncol == [0, 0]
    # the context stays usable
    cols, st, rounds, ncol = bg.bgpc_color_batched(ctx, [other, clique])
    check_against_oracle([gg.random_bipartite(200, 100, 3, seed=1),
                          gg.from_nets(40, [list(range(40))])], cols, rounds, ncol)
