"""GPU parity: the CUDA path, called through the C ABI, against the CPU
oracle on the same seeded inputs.  Colors, round counts, |W_r| and the
traversed two-hop entries per round must match bit for bit."""
import numpy as np
import pytest
import torch

import graphgen as gg
import hubrule
import oracle as O

pytestmark = pytest.mark.gpu

POLICIES = [O.FF, O.B1, O.B2, O.B2X]


@pytest.fixture(scope="module")
def bg():
    import paper_1701_02628_gb300 as m
    from paper_1701_02628_gb300 import build
    build.build()
    return m


@pytest.fixture(scope="module")
def ctx(bg):
    return bg.Context(0)


def run_gpu(bg, ctx, g, **kw):
    dg = bg.DeviceGraph.from_host(g, "cuda:0")
    rank = kw.pop("rank", None)
    if rank is not None:
        kw["rank"] = torch.as_tensor(rank, dtype=torch.int32, device="cuda:0")
    colors, st, rc = bg.bgpc_color(ctx, dg, **kw)
    torch.cuda.synchronize()
    return colors.cpu().numpy(), st, rc, dg


def assert_parity(bg, ctx, g, policy=O.FF, chunk=64, waves=16, big_net=64, rank=None,
                  net_rounds=0, **kw):
    ref = O.rs_color(g, policy, chunk=chunk, waves=waves, big_net=big_net, rank=rank,
                     nthreads=8, net_rounds=net_rounds)
    assert ref.status == O.OK
    got, st, rc, dg = run_gpu(bg, ctx, g, policy=policy, chunk=chunk, waves=waves,
                              big_net=big_net, rank=rank, validate=True,
                              net_rounds=net_rounds, **kw)
    assert rc == bg.BGPC_OK
    bad = np.nonzero(got != ref.colors)[0]
    assert bad.size == 0, f"{bad.size} colors differ, first at {bad[:8]}"
    assert st["rounds"] == ref.rounds
    assert st["w_per_round"] == ref.w_per_round.tolist()[:64]
    assert st["trav_per_round"] == ref.trav_per_round.tolist()[:64]
    assert st["colors"] == int(ref.colors.max()) + 1
    assert bg.bgpc_validate(ctx, dg, torch.as_tensor(got, device="cuda:0")) == 0
    return st


# ------------------------------------------------------------------ configs

def test_config1_random_2000(bg, ctx):
    g = gg.random_bipartite(2000, 2000, 5, seed=1)
    st = assert_parity(bg, ctx, g)
    assert st["w_per_round"][0] == 2000


@pytest.mark.parametrize("policy", POLICIES)
def test_policies_random(bg, ctx, policy):
    g = gg.random_bipartite(5000, 3000, 6, seed=21)
    assert_parity(bg, ctx, g, policy=policy)


@pytest.mark.parametrize("policy", POLICIES)
def test_policies_stencil(bg, ctx, policy):
    assert_parity(bg, ctx, gg.stencil9(96), policy=policy)


@pytest.mark.parametrize("policy", POLICIES)
def test_policies_power_law(bg, ctx, policy):
    """Small Chung-Lu graph: hub nets above T (reverse first fit) and large
    two-hop volumes (the CTA-wide byte-map path)."""
    g = gg.chung_lu(20000, 16, 1500, 2.1, seed=4)
    assert_parity(bg, ctx, g, policy=policy)


def hub_graph():
    """Three nets above the smallest hub threshold (512 members), overlapping, plus
    2500 small random nets: the members of a hub net gather it from its
    color bitmap and find their chunk-mates in it by binary search."""
    rng = np.random.default_rng(4)
    nets = [list(range(0, 1500)), list(range(500, 3000)), list(rng.choice(3000, 1100, replace=False))]
    nets += [list(rng.choice(3000, rng.integers(2, 40), replace=False)) for _ in range(2500)]
    return gg.from_nets(3000, [sorted(set(int(x) for x in n)) for n in nets])


@pytest.mark.parametrize("policy", POLICIES)
def test_hub_nets(bg, ctx, policy):
    g = hub_graph()
    st = assert_parity(bg, ctx, g, policy=policy)
    assert st["hub_pairs"] > 0 and st["trav_hub"] > 0
    assert hubrule.check(st, np.diff(g.b_ptr)) == 512
    # 47 nets above 512 members; in its third round (537 vertices) the chunks
    # spread over more than 2048 ids, so 83 vertices find their hub
    # chunk-mates pair by pair instead of from the hubs' member windows
    g = gg.chung_lu(30000, 12, 6000, 2.1, seed=3)
    st = assert_parity(bg, ctx, g, policy=policy)
    assert st["hub_pairs"] > 0
    assert hubrule.check(st, np.diff(g.b_ptr)) == 512 and st["hubs"] > 0


@pytest.mark.parametrize("policy", [O.FF, O.B2])
def test_hub_nets_rank_and_small_chunks(bg, ctx, policy):
    g = hub_graph()
    rank = np.random.default_rng(9).permutation(g.n_a).astype(np.int32)
    assert_parity(bg, ctx, g, policy=policy, rank=rank)
    assert_parity(bg, ctx, g, policy=policy, chunk=5, waves=7, big_net=300)


@pytest.mark.parametrize("policy", [O.FF, O.B2X])
@pytest.mark.parametrize("detect", [1, 2, 0])
def test_detect_tiers(bg, ctx, policy, detect):
    """Conflict detection after the first round scans every net (1), looks
    up only the (W member, net) pairs in a hash table (2) or picks one of
    them by the size of W (0): a mapping choice, the oracle's colors always."""
    for g in (hub_graph(), gg.chung_lu(20000, 16, 1500, 2.1, seed=4),
              gg.random_bipartite(3000, 400, 9, seed=6)):
        assert_parity(bg, ctx, g, policy=policy, detect=detect)
    g = gg.from_nets(40, [list(range(40))])  # a clique: one round per vertex
    st = assert_parity(bg, ctx, g, policy=policy, chunk=1, waves=1, big_net=O.NO_BIG,
                       detect=detect)
    assert st["rounds"] == 40


@pytest.mark.parametrize("policy", [O.FF, O.B2])
def test_gather_cta_form(bg, ctx, policy):
    """The CTA-per-piece gather (taken by itself only for color bounds above
    ~110k colors, where eight warp bitmaps no longer fit in shared memory),
    forced on small graphs: hub nets, multi-piece vertices, rank order."""
    g = hub_graph()
    assert_parity(bg, ctx, g, policy=policy, gather=1)
    rank = np.random.default_rng(9).permutation(g.n_a).astype(np.int32)
    assert_parity(bg, ctx, g, policy=policy, rank=rank, gather=1)
    g = gg.chung_lu(20000, 16, 1500, 2.1, seed=4)
    assert_parity(bg, ctx, g, policy=policy, gather=1)
    g = gg.from_nets(3000, [list(range(3000))])
    assert_parity(bg, ctx, g, policy=policy, gather=1)


@pytest.mark.parametrize("chunk,waves,big_net", [(1, 1, O.NO_BIG), (7, 3, 2), (32, 16, 0),
                                                 (64, 1, 8), (64, 64, O.NO_BIG), (13, 5, 64)])
def test_semantic_parameters(bg, ctx, chunk, waves, big_net):
    g = gg.chung_lu(6000, 10, 600, 2.1, seed=8)
    assert_parity(bg, ctx, g, chunk=chunk, waves=waves, big_net=big_net)


@pytest.mark.parametrize("policy", [O.FF, O.B1, O.B2])
def test_rank_order(bg, ctx, policy):
    g = gg.random_bipartite(4000, 2500, 7, seed=5)
    rank = np.random.default_rng(3).permutation(g.n_a).astype(np.int32)
    assert_parity(bg, ctx, g, policy=policy, rank=rank)


@pytest.mark.parametrize("seed", range(24))
def test_fuzz_small_graphs(bg, ctx, seed):
    """Sizes 1..5000, skewed degrees, empty nets, isolated vertices, giant nets."""
    rng = np.random.default_rng(1000 + seed)
    n_a = int(rng.integers(1, 5000))
    n_b = int(rng.integers(1, 3000))
    kind = seed % 4
    nets = []
    for v in range(n_b):
        if kind == 0:
            s = int(rng.integers(0, 6))
        elif kind == 1:
            s = int(min(n_a, rng.pareto(1.2) * 2))
        elif kind == 2:
            s = int(rng.integers(0, 3)) if v else n_a  # one giant net
        else:
            s = int(rng.integers(0, min(n_a, 40) + 1))
        nets.append(rng.choice(n_a, size=min(s, n_a), replace=False))
    g = gg.from_nets(n_a, nets)
    policy = int(rng.integers(0, 4))
    chunk = int(rng.choice([1, 5, 32, 64]))
    waves = int(rng.choice([1, 2, 16]))
    big_net = int(rng.choice([0, 4, 64, O.NO_BIG]))
    assert_parity(bg, ctx, g, policy=policy, chunk=chunk, waves=waves, big_net=big_net)


# ------------------------------------------------------------------- D2GC

@pytest.mark.parametrize("policy", POLICIES)
def test_d2gc_rmat_small(bg, ctx, policy):
    ug = gg.rmat(12, 16, seed=3)
    ref = O.rs_color(O.closed_nbhd(ug), policy, nthreads=8)
    dug = bg.DeviceUGraph.from_host(ug, "cuda:0")
    colors, st, rc = bg.d2gc_color(ctx, dug, policy=policy, validate=True)
    got = colors.cpu().numpy()
    assert np.array_equal(got, ref.colors)
    assert st["rounds"] == ref.rounds
    assert st["w_per_round"] == ref.w_per_round.tolist()[:64]
    assert O.d2_conflicts(ug, got) == 0


def test_d2gc_closed_forms(bg, ctx):
    for edges, n, want in [([(i, i + 1) for i in range(9)], 10, None),
                           ([(0, i) for i in range(1, 7)], 7, list(range(7)))]:
        ug = gg.from_edges(n, edges)
        dug = bg.DeviceUGraph.from_host(ug, "cuda:0")
        colors, st, _ = bg.d2gc_color(ctx, dug, chunk=n, waves=1, big_net=bg.NO_BIG)
        got = colors.cpu().numpy().tolist()
        assert got == (want if want is not None else [i % 3 for i in range(n)])


# ------------------------------------------------------------- edge cases

def test_empty_and_degenerate(bg, ctx):
    # no vertices
    g = gg.from_nets(0, [])
    got, st, rc, _ = run_gpu(bg, ctx, g)
    assert rc == 0 and got.size == 0 and st["rounds"] == 0
    # vertices without nets -> all 0 in one round
    g = gg.from_nets(100, [[], [], []])
    got, st, rc, _ = run_gpu(bg, ctx, g)
    assert got.tolist() == [0] * 100 and st["rounds"] == 1
    # one vertex
    g = gg.from_nets(1, [[0]])
    got, st, rc, _ = run_gpu(bg, ctx, g)
    assert got.tolist() == [0]


def test_giant_clique_net(bg, ctx):
    """One net holding every vertex forces n distinct colors; with T below its
    size every vertex takes the reverse first-fit color (shifted by the colors
    its earlier chunk-mates took)."""
    n = 3000
    g = gg.from_nets(n, [list(range(n))])
    st = assert_parity(bg, ctx, g)
    assert st["colors"] >= n
    st = assert_parity(bg, ctx, g, big_net=O.NO_BIG, chunk=64, waves=4)
    assert st["colors"] >= n


def test_errors(bg, ctx):
    g = gg.random_bipartite(300, 200, 4, seed=2)
    dg = bg.DeviceGraph.from_host(g, "cuda:0")
    with pytest.raises(bg.BgpcError) as e:
        bg.bgpc_color(ctx, dg, chunk=65)
    assert e.value.status == bg.BGPC_EINVAL
    with pytest.raises(bg.BgpcError) as e:
        bg.bgpc_color(ctx, dg, waves=0)
    assert e.value.status == bg.BGPC_EINVAL
    for d in (-1, 3):
        with pytest.raises(bg.BgpcError) as e:
            bg.bgpc_color(ctx, dg, detect=d)
        assert e.value.status == bg.BGPC_EINVAL
    for v in (-1, 2):
        with pytest.raises(bg.BgpcError) as e:
            bg.bgpc_color(ctx, dg, gather=v)
        assert e.value.status == bg.BGPC_EINVAL
    bad_rank = torch.zeros(g.n_a, dtype=torch.int32, device="cuda:0")
    with pytest.raises(bg.BgpcError) as e:
        bg.bgpc_color(ctx, dg, rank=bad_rank, validate=True)
    assert e.value.status == bg.BGPC_EINVAL
    # unsorted adjacency
    a_idx = dg.a_idx.clone()
    a_idx[0], a_idx[1] = dg.a_idx[1].item(), dg.a_idx[0].item()
    bad = bg.DeviceGraph(dg.n_a, dg.n_b, dg.a_ptr, a_idx, dg.b_ptr, dg.b_idx)
    with pytest.raises(bg.BgpcError) as e:
        bg.bgpc_color(ctx, bad, validate=True)
    assert e.value.status == bg.BGPC_EUNSORTED
    # CSR and CSC disagree (an entry moved to another net)
    a_idx = dg.a_idx.clone()
    row = g.a_idx[g.a_ptr[0]:g.a_ptr[1]]
    free = [v for v in range(g.n_b) if v not in set(row.tolist()) and v > row[-1]]
    a_idx[g.a_ptr[1] - 1] = free[0]
    bad = bg.DeviceGraph(dg.n_a, dg.n_b, dg.a_ptr, a_idx, dg.b_ptr, dg.b_idx)
    with pytest.raises(bg.BgpcError) as e:
        bg.bgpc_color(ctx, bad, validate=True)
    assert e.value.status == bg.BGPC_EUNSORTED
    # CSR and CSC each sorted and in range but holding different pairs (one
    # member of a net swapped for a vertex outside it, in both directions of
    # the row order): the validation's pair check
    v = int(np.argmax(np.diff(g.b_ptr)))
    members = set(g.b_idx[g.b_ptr[v]:g.b_ptr[v + 1]].tolist())
    w_out = next(u for u in range(g.n_a) if u not in members)
    lst = sorted((members - {int(g.b_idx[g.b_ptr[v]])}) | {w_out})
    b_idx = dg.b_idx.clone()
    b_idx[g.b_ptr[v]:g.b_ptr[v + 1]] = torch.as_tensor(lst, dtype=torch.int32, device="cuda:0")
    bad = bg.DeviceGraph(dg.n_a, dg.n_b, dg.a_ptr, dg.a_idx, dg.b_ptr, b_idx)
    with pytest.raises(bg.BgpcError) as e:
        bg.bgpc_color(ctx, bad, validate=True)
    assert e.value.status == bg.BGPC_EUNSORTED
    # index out of range
    a_idx = dg.a_idx.clone()
    a_idx[g.a_ptr[1] - 1] = g.n_b + 5
    bad = bg.DeviceGraph(dg.n_a, dg.n_b, dg.a_ptr, a_idx, dg.b_ptr, dg.b_idx)
    with pytest.raises(bg.BgpcError) as e:
        bg.bgpc_color(ctx, bad, validate=True)
    assert e.value.status == bg.BGPC_EINVAL
    # round cap: a clique under the Jacobi reading needs s rounds
    clique = bg.DeviceGraph.from_host(gg.from_nets(40, [list(range(40))]), "cuda:0")
    with pytest.raises(bg.BgpcError) as e:
        bg.bgpc_color(ctx, clique, chunk=1, waves=1, big_net=bg.NO_BIG, max_rounds=5)
    assert e.value.status == bg.BGPC_EROUNDS
    # wall-clock limit: a clique under the Jacobi reading takes 40 rounds; a
    # 1 us limit has passed by the first wait for the device (after the setup)
    with pytest.raises(bg.BgpcError) as e:
        bg.bgpc_color(ctx, clique, chunk=1, waves=1, big_net=bg.NO_BIG, timeout_us=1)
    assert e.value.status == bg.BGPC_ETIMEOUT
    with pytest.raises(bg.BgpcError) as e:
        bg.bgpc_color(ctx, dg, timeout_us=-1)
    assert e.value.status == bg.BGPC_EINVAL
    _, st, rc = bg.bgpc_color(ctx, clique, chunk=1, waves=1, big_net=bg.NO_BIG,
                              timeout_us=60_000_000)
    assert rc == bg.BGPC_OK and st["rounds"] == 40 and st["ms_total"] > 0
    # the context stays usable after errors
    assert_parity(bg, ctx, g)


def test_color_sets(bg, ctx):
    g = gg.random_bipartite(3000, 2000, 5, seed=9)
    for pol in POLICIES:
        got, st, _, _ = run_gpu(bg, ctx, g, policy=pol, want_balance=True)
        ref = O.balance(got)
        assert st["n_sets"] == ref["colors"] and st["max_card"] == ref["max_card"]
        assert abs(st["mean_card"] - ref["mean_card"]) < 1e-9
        assert abs(st["std_card"] - ref["std_card"]) < 1e-9 * max(1.0, ref["std_card"])
        card, s2 = bg.bgpc_color_sets(ctx, torch.as_tensor(got, device="cuda:0"), st["colors"])
        K, rc = O.color_sets(got)
        assert np.array_equal(card.cpu().numpy(), rc)


def test_validate_counts_conflicts(bg, ctx):
    g = gg.chung_lu(5000, 12, 800, 2.1, seed=6)
    got, st, _, dg = run_gpu(bg, ctx, g)
    bad = got.copy()
    rng = np.random.default_rng(0)
    bad[rng.choice(g.n_a, 50, replace=False)] = 0
    bad[:3] = -1
    assert bg.bgpc_validate(ctx, dg, torch.as_tensor(bad, device="cuda:0")) == O.conflicts(g, bad)


# ------------------------------------------------------ wave-by-wave state

def test_wave_snapshots_match(bg, ctx):
    """The state at the start of every wave (colors and work queue) equals
    the oracle's, on a graph with several rounds."""
    g = gg.chung_lu(12000, 16, 1200, 2.1, seed=12)
    C, Q, T = 32, 4, 16
    full = O.rs_color(g, O.B2, chunk=C, waves=Q, big_net=T)
    dg = bg.DeviceGraph.from_host(g, "cuda:0")
    W_out = torch.empty(g.n_a, dtype=torch.int32, device="cuda:0")
    for wv in range(1, full.rounds * Q):
        ref = O.rs_color(g, O.B2, chunk=C, waves=Q, big_net=T, stop_after_waves=wv)
        colors, st, rc = bg.bgpc_color(ctx, dg, policy=O.B2, chunk=C, waves=Q, big_net=T,
                                       stop_after_waves=wv, W_out=W_out)
        assert rc == bg.BGPC_STOPPED and ref.status == O.STOPPED
        assert st["stopped_m"] == ref.m and st["stopped_wave"] == ref.wave
        assert np.array_equal(colors.cpu().numpy(), ref.colors)
        assert np.array_equal(W_out[:ref.m].cpu().numpy(), ref.W)


# ------------------------------------------------- net-based first round (N1)

@pytest.mark.parametrize("policy", POLICIES)
def test_net_round_parity(bg, ctx, policy):
    """N1-*: the first round colored net by net (Alg. 8), the later rounds by
    vertex waves; colors, rounds, |W_r| and traversal equal the oracle's."""
    rng = np.random.default_rng(71)
    graphs = [gg.random_bipartite(2000, 2000, 5, seed=1), gg.stencil9(64),
              gg.chung_lu(20000, 16, 1500, 2.1, seed=4), hub_graph(),
              gg.from_nets(7, [[0, 1, 2], [], [2, 4], [5]]),      # isolated vertices 3 and 6
              gg.from_nets(40, [list(range(40))])]
    for g in graphs:
        assert_parity(bg, ctx, g, policy=policy, net_rounds=1)
    g = gg.chung_lu(20000, 16, 1500, 2.1, seed=4)
    rank = rng.permutation(g.n_a).astype(np.int32)
    assert_parity(bg, ctx, g, policy=policy, net_rounds=1, rank=rank)
    assert_parity(bg, ctx, g, policy=policy, net_rounds=1, chunk=7, waves=5, big_net=20)
    for d in (1, 2):
        assert_parity(bg, ctx, hub_graph(), policy=policy, net_rounds=1, detect=d)


def test_net_round_tentative_colors(bg, ctx):
    """Stopped before its conflict removal, the net round's tentative colors
    and work queue equal the oracle's (a net round counts as one wave)."""
    for g in (gg.chung_lu(20000, 16, 1500, 2.1, seed=4), gg.stencil9(50)):
        ref = O.rs_color(g, net_rounds=1, stop_after_waves=1, stop_before_removal=True)
        assert ref.status == O.STOPPED and ref.wave == 1
        W = torch.empty(g.n_a, dtype=torch.int32, device="cuda:0")
        got, st, rc, _ = run_gpu(bg, ctx, g, net_rounds=1, stop_after_waves=1,
                                 stop_before_removal=True, W_out=W)
        assert rc == bg.BGPC_STOPPED and st["stopped_wave"] == 1
        assert np.array_equal(got, ref.colors)
        assert np.array_equal(W[:st["stopped_m"]].cpu().numpy(), ref.W)
        # one wave later: the first vertex-based wave of round 2
        ref2 = O.rs_color(g, net_rounds=1, stop_after_waves=2)
        got2, st2, rc2, _ = run_gpu(bg, ctx, g, net_rounds=1, stop_after_waves=2)
        assert rc2 == bg.BGPC_STOPPED and np.array_equal(got2, ref2.colors)


@pytest.mark.parametrize("policy", [O.FF, O.B1, O.B2])
def test_net_round_d2gc(bg, ctx, policy):
    """D2GC with the net-based first round in Alg. 9's order (the center of
    N[v] first)."""
    for ug in (gg.rmat(12, 16, seed=3), gg.from_edges(4, [(2, 0), (2, 1), (2, 3)])):
        cn = O.closed_nbhd(ug)
        ref = O.rs_color(cn, policy, net_rounds=1, center_first=True, nthreads=8)
        dug = bg.DeviceUGraph.from_host(ug, "cuda:0")
        got, st, rc = bg.d2gc_color(ctx, dug, policy=policy, net_rounds=1)
        assert rc == bg.BGPC_OK
        assert np.array_equal(got.cpu().numpy(), ref.colors)
        assert st["rounds"] == ref.rounds and st["w_per_round"] == ref.w_per_round.tolist()
        assert O.d2_conflicts(ug, got.cpu().numpy()) == 0


def test_net_rounds_limit(bg, ctx):
    """Only the first round can be net-based on the GPU (N1-*)."""
    dg = bg.DeviceGraph.from_host(gg.random_bipartite(300, 200, 4, seed=2), "cuda:0")
    for nr in (-1, 2):
        with pytest.raises(bg.BgpcError) as e:
            bg.bgpc_color(ctx, dg, net_rounds=nr)
        assert e.value.status == bg.BGPC_EINVAL
