"""Pins for the CPU oracle: facts fixed by the paper and by mathematics, not
by the oracle itself (closed forms, exhaustive search, invariants, reductions,
hand-derived fixtures in tests/golden/, an independent Python statement).

Section / algorithm numbers refer to Tas, Kaya, Saule, arXiv 1701.02628.
"""
import json
import os

import numpy as np
import pytest

import graphgen as gg
import oracle as O
import rs_py

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
POLICIES = [O.FF, O.B1, O.B2, O.B2X]
NAMES = {O.FF: "FF", O.B1: "B1", O.B2: "B2", O.B2X: "B2X"}


def golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def nets_of(g):
    return [g.b_idx[g.b_ptr[v]:g.b_ptr[v + 1]].tolist() for v in range(g.n_b)]


def random_tiny(rng, n_a, n_b, pmax):
    nets = []
    for _ in range(n_b):
        s = int(rng.integers(0, min(pmax, n_a) + 1))
        nets.append(sorted(rng.choice(n_a, size=s, replace=False).tolist()))
    return gg.from_nets(n_a, nets), nets


# --------------------------------------------------------------- closed forms

@pytest.mark.parametrize("n", [3, 4, 7, 12, 64])
def test_stencil_first_fit_closed_form(n):
    """9-point stencil Jacobian, natural order: first fit gives
    c(i, j) = 3 (i mod 3) + (j mod 3) (two columns conflict iff |di|,|dj| <= 2)."""
    g = gg.stencil9(n)
    i, j = np.divmod(np.arange(n * n), n)
    assert np.array_equal(O.seq_color(g), 3 * (i % 3) + (j % 3))


def test_single_net_is_a_clique():
    """One net of size s: every pair conflicts, first fit gives 0..s-1."""
    for s in [1, 2, 5, 33]:
        g = gg.from_nets(s, [list(range(s))])
        assert O.seq_color(g).tolist() == list(range(s))
        if s <= 20:
            assert O.bruteforce_min(g) == s


def test_disjoint_nets_use_max_net_size_colors():
    sizes = [3, 7, 1, 5]
    nets, base = [], 0
    for s in sizes:
        nets.append(list(range(base, base + s)))
        base += s
    g = gg.from_nets(base, nets)
    c = O.seq_color(g)
    assert c.max() + 1 == max(sizes)
    assert O.conflicts(g, c) == 0


def test_no_two_hop_edges_all_zero():
    """Nets of size <= 1 and isolated vertices: F is always empty."""
    g = gg.from_nets(6, [[0], [], [3], [5]])
    assert O.seq_color(g).tolist() == [0] * 6
    r = O.rs_color(g, chunk=1, waves=1)
    assert r.rounds == 1 and r.colors.tolist() == [0] * 6


def test_d2gc_closed_forms():
    """D2GC through N[u] nets (Sec. IV): path -> i mod 3; star K_{1,m} ->
    0..m; cycle C7 -> [0,1,2,0,1,2,3]."""
    n = 10
    path = gg.from_edges(n, [(i, i + 1) for i in range(n - 1)])
    assert O.seq_color(O.closed_nbhd(path)).tolist() == [i % 3 for i in range(n)]
    m = 6
    star = gg.from_edges(m + 1, [(0, i) for i in range(1, m + 1)])
    assert O.seq_color(O.closed_nbhd(star)).tolist() == list(range(m + 1))
    c7 = gg.from_edges(7, [(i, (i + 1) % 7) for i in range(7)])
    assert O.seq_color(O.closed_nbhd(c7)).tolist() == [0, 1, 2, 0, 1, 2, 3]


def test_closed_nbhd_structure():
    g = gg.from_edges(5, [(0, 3), (1, 3), (3, 4)])
    cn = O.closed_nbhd(g)
    lists = [cn.a_idx[cn.a_ptr[u]:cn.a_ptr[u + 1]].tolist() for u in range(5)]
    assert lists == [[0, 3], [1, 3], [2], [0, 1, 3, 4], [3, 4]]


# ------------------------------------------------------------- brute force

def test_bruteforce_known_values():
    """Chromatic numbers of small conflict graphs: nets = edges of C5 -> 3,
    C6 -> 2, K4 -> 4, no nets -> 1."""
    c5 = gg.from_nets(5, [[i, (i + 1) % 5] for i in range(5)])
    c6 = gg.from_nets(6, [[i, (i + 1) % 6] for i in range(6)])
    k4 = gg.from_nets(4, [[0, 1, 2, 3]])
    empty = gg.from_nets(3, [])
    assert [O.bruteforce_min(g) for g in (c5, c6, k4, empty)] == [3, 2, 4, 1]


@pytest.mark.parametrize("seed", range(12))
def test_greedy_never_beats_optimum_and_is_valid(seed):
    rng = np.random.default_rng(seed)
    g, _ = random_tiny(rng, int(rng.integers(2, 10)), int(rng.integers(1, 8)), 4)
    opt = O.bruteforce_min(g)
    for pol in POLICIES:
        c = O.seq_color(g, pol)
        assert O.conflicts(g, c) == 0
        assert c.max() + 1 >= opt
        r = O.rs_color(g, pol, chunk=2, waves=2, big_net=2)
        assert r.status == O.OK and O.conflicts(g, r.colors) == 0
        assert r.colors.max() + 1 >= opt


def test_d2gc_valid_by_direct_distance_definition():
    """Colorings from N[u] nets are valid for the shortest-path definition
    of D2GC (Sec. II), checked by a direct depth-2 walk."""
    ug = gg.rmat(9, 8, seed=5)
    cn = O.closed_nbhd(ug)
    for pol in POLICIES:
        assert O.d2_conflicts(ug, O.seq_color(cn, pol)) == 0
        r = O.rs_color(cn, pol, chunk=8, waves=4, big_net=16)
        assert r.status == O.OK and O.d2_conflicts(ug, r.colors) == 0
    bad = O.seq_color(cn).copy()
    nb = ug.idx[ug.ptr[0]:ug.ptr[1]]
    if len(nb) >= 2:  # two neighbours of vertex 0 are at distance 2
        bad[nb[1]] = bad[nb[0]]
        assert O.d2_conflicts(ug, bad) > 0


# ---------------------------------------------------------- greedy bound

@pytest.mark.parametrize("pol", POLICIES)
def test_greedy_bound(pol):
    """#colors <= max_w |nbor(w)| + 1 for every policy; first fit also has
    c[w] <= |nbor(w)| per vertex (Alg. 2 picks the smallest of |F|+1 colors)."""
    g = gg.random_bipartite(500, 300, 4, seed=7)
    best, sizes = O.max_nbor(g)
    c = O.seq_color(g, pol)
    assert c.max() <= best
    r = O.rs_color(g, pol, chunk=16, waves=4, big_net=8)
    assert r.colors.max() <= best
    if pol == O.FF:
        assert np.all(c <= sizes) and np.all(r.colors <= sizes)


# ------------------------------------------------------ RS reductions

@pytest.mark.parametrize("pol", POLICIES)
def test_rs_with_one_chunk_is_sequential(pol):
    """RS(C >= |V_A|, any Q, T = inf) is the sequential greedy, bit-exact."""
    g = gg.random_bipartite(300, 200, 5, seed=3)
    rank = np.random.default_rng(1).permutation(g.n_a).astype(np.int32)
    for Q in (1, 3, 16):
        r = O.rs_color(g, pol, chunk=g.n_a, waves=Q, big_net=O.NO_BIG)
        assert r.rounds == 1
        assert np.array_equal(r.colors, O.seq_color(g, pol))
        r = O.rs_color(g, pol, chunk=g.n_a + 5, waves=Q, big_net=O.NO_BIG, rank=rank)
        assert np.array_equal(r.colors, O.seq_color(g, pol, rank=rank))


def test_rs_jacobi_on_a_clique_takes_s_rounds():
    """RS(1, 1, inf) is the literal Jacobi reading: on one net of size s all
    members pick the same first-fit color each round and only the lowest rank
    keeps it, so there are s rounds and c[u_i] = i."""
    s = 9
    g = gg.from_nets(s, [list(range(s))])
    r = O.rs_color(g, O.FF, chunk=1, waves=1, big_net=O.NO_BIG)
    assert r.rounds == s and r.colors.tolist() == list(range(s))
    assert r.w_per_round.tolist() == list(range(s, 0, -1))


def test_rs_round_count_bound_and_first_vertex_survives():
    g = gg.random_bipartite(400, 50, 6, seed=11)
    r = O.rs_color(g, O.FF, chunk=1, waves=1, big_net=O.NO_BIG)
    assert r.status == O.OK and r.rounds <= g.n_a
    assert np.all(np.diff(r.w_per_round) < 0)  # the lowest-rank W vertex always keeps its color


def test_rs_round_cap():
    g = gg.from_nets(6, [list(range(6))])
    r = O.rs_color(g, O.FF, chunk=1, waves=1, big_net=O.NO_BIG, max_rounds=3)
    assert r.status == O.EROUNDS


def test_rs_thread_count_invariance():
    g = gg.chung_lu(20000, 16, 1500, 2.1, seed=4)
    base = O.rs_color(g, O.B2, chunk=64, waves=16, big_net=64, nthreads=1)
    for t in (2, 3, 8):
        r = O.rs_color(g, O.B2, chunk=64, waves=16, big_net=64, nthreads=t)
        assert np.array_equal(r.colors, base.colors)
        assert np.array_equal(r.w_per_round, base.w_per_round)


def test_traversal_of_round_one_is_e2():
    """Round 1 traverses sum_v |vtxs(v)| (|vtxs(v)| - 1) two-hop entries,
    the cost of one vertex-based sweep (Sec. III)."""
    g = gg.random_bipartite(2000, 2000, 5, seed=1)
    s = np.diff(g.b_ptr).astype(np.int64)
    r = O.rs_color(g)
    assert r.trav_per_round[0] == int((s * (s - 1)).sum())
    assert r.w_per_round[0] == g.n_a


# ---------------------------------------------------------- golden fixtures

@pytest.mark.parametrize("name", ["rs_overlay_waves.json", "rs_reverse_first_fit.json",
                                  "rs_reverse_fallback.json"])
def test_golden_rs(name):
    fx = golden(name)
    g = gg.from_nets(fx["n_a"], fx["nets"])
    p = fx["params"]
    r = O.rs_color(g, p["policy"], chunk=p["chunk"], waves=p["waves"], big_net=p["big_net"])
    e = fx["expected"]
    assert r.status == O.OK
    assert r.colors.tolist() == e["colors"]
    assert r.rounds == e["rounds"]
    assert r.w_per_round.tolist() == e["w_per_round"]
    assert r.trav_per_round.tolist() == e["trav_per_round"]
    c_py, hist = rs_py.rs(fx["n_a"], fx["nets"], p["policy"], p["chunk"], p["waves"], p["big_net"])
    assert c_py == e["colors"] and hist == e["w_per_round"]


def test_golden_sequential_balancing():
    fx = golden("seq_balancing.json")
    g = gg.from_nets(fx["n_a"], fx["nets"])
    for pol in POLICIES:
        assert O.seq_color(g, pol).tolist() == fx["expected"][NAMES[pol]]
        assert rs_py.seq(fx["n_a"], fx["nets"], pol) == fx["expected"][NAMES[pol]]


def test_golden_chunk_state():
    fx = golden("rs_chunk_state.json")
    g = gg.from_nets(fx["n_a"], fx["nets"])
    for pname, pol in (("B1", O.B1), ("B2", O.B2), ("FF", O.FF)):
        out = O.rs_chunks(g, fx["S"], fx["W"], fx["chunks"], pol,
                          chunk=fx["params"]["chunk"], big_net=fx["params"]["big_net"])
        assert out.tolist() == fx["expected"][pname]


def test_balance_statistics():
    c = np.array([0, 1, 2, 0, 2, 0], np.int32)
    K, card = O.color_sets(c)
    assert K == 3 and card.tolist() == [3, 1, 2]
    b = O.balance(c)
    assert b["max_card"] == 3 and b["mean_card"] == 2.0
    assert abs(b["std_card"] - np.std([3, 1, 2])) < 1e-12
    K, card = O.color_sets(np.array([4, 4, 0], np.int32))
    assert K == 2 and card.tolist() == [1, 0, 0, 0, 2]


# ------------------------------------- independent Python statement of RS

@pytest.mark.parametrize("seed", range(40))
def test_rs_matches_independent_python(seed):
    rng = np.random.default_rng(100 + seed)
    n_a = int(rng.integers(1, 40))
    g, nets = random_tiny(rng, n_a, int(rng.integers(0, 25)), 12)
    pol = int(rng.integers(0, 4))
    C = int(rng.integers(1, 9))
    Q = int(rng.integers(1, 5))
    T = int(rng.choice([1, 2, 4, 8, O.NO_BIG]))
    rank = rng.permutation(n_a).astype(np.int32) if seed % 3 == 0 else None
    r = O.rs_color(g, pol, chunk=C, waves=Q, big_net=T, rank=rank)
    c_py, hist = rs_py.rs(n_a, nets, pol, C, Q, T, None if rank is None else rank.tolist())
    assert r.status == O.OK
    assert r.colors.tolist() == c_py
    assert r.w_per_round.tolist() == hist
    assert O.seq_color(g, pol, rank=rank).tolist() == rs_py.seq(
        n_a, nets, pol, None if rank is None else rank.tolist())


# -------------------------------- wave stepping (used by full-size parity)

def test_wave_stepping_reproduces_full_run():
    """Stopping after each wave and recoloring that wave's chunks with
    rs_chunks, then applying the conflict rule, reproduces the full run."""
    g = gg.random_bipartite(700, 500, 5, seed=9)
    C, Q, T, pol = 16, 4, 6, O.B1
    full = O.rs_color(g, pol, chunk=C, waves=Q, big_net=T)
    total_waves = full.rounds * Q
    for wv in range(1, total_waves):
        st = O.rs_color(g, pol, chunk=C, waves=Q, big_net=T, stop_after_waves=wv)
        assert st.status == O.STOPPED
        nxt = O.rs_color(g, pol, chunk=C, waves=Q, big_net=T, stop_after_waves=wv + 1)
        nch = (st.m + C - 1) // C
        q = st.wave
        chunks = [j for j in range(nch) if rs_py.wave_of(j, Q) == q]
        out = O.rs_chunks(g, st.colors, st.W, chunks, pol, chunk=C, big_net=T)
        pos = [p for j in chunks for p in range(j * C, min(st.m, (j + 1) * C))]
        if nxt.status == O.STOPPED and nxt.wave == q + 1:
            assert np.array_equal(out[pos], nxt.colors[st.W[pos]])
    # conflict rule on the last round's colors
    st = O.rs_color(g, pol, chunk=C, waves=Q, big_net=T, stop_after_waves=Q - 1)
    nch = (st.m + C - 1) // C
    chunks = [j for j in range(nch) if rs_py.wave_of(j, Q) == Q - 1]
    out = O.rs_chunks(g, st.colors, st.W, chunks, pol, chunk=C, big_net=T)
    c = st.colors.copy()
    for j in chunks:
        for p in range(j * C, min(st.m, (j + 1) * C)):
            c[st.W[p]] = out[p]
    lose, rc = O.rs_losers(g, c, st.W, np.arange(st.m))
    assert rc == O.OK
    r2 = O.rs_color(g, pol, chunk=C, waves=Q, big_net=T, stop_after_waves=Q)
    if r2.status == O.STOPPED:
        assert np.array_equal(r2.W, st.W[lose.astype(bool)])


# ------------------------------------------- validity counts and nbor sizes
#
# orc_conflicts, orc_d2_conflicts and orc_max_nbor underlie every validity
# check and the greedy bound above, so they are pinned on hand-counted cases
# and against the conflict graph written as an incidence-matrix product
# (u ~ w iff row u and row w of the n_a x n_b incidence matrix B share a
# column, i.e. (B B^T)[u, w] > 0 for u != w: Sec. II's definition of BGPC).

def conflict_matrix(g):
    B = np.zeros((g.n_a, g.n_b), np.int64)
    rows = np.repeat(np.arange(g.n_a), np.diff(g.a_ptr))
    B[rows, g.a_idx] = 1
    M = (B @ B.T) > 0
    np.fill_diagonal(M, False)
    return M


def test_conflicts_hand_counts():
    """Counts of vertices that are uncolored or clash, derived by hand."""
    g = gg.from_nets(4, [[0, 1, 2, 3]])
    assert O.conflicts(g, [0, 0, 1, 1]) == 4     # two clashing pairs
    assert O.conflicts(g, [0, 1, 2, 2]) == 2     # one clashing pair
    assert O.conflicts(g, [0, 1, 2, 3]) == 0
    assert O.conflicts(g, [-1, 1, 2, 3]) == 1    # uncolored counts
    assert O.conflicts(g, [-1, -1, 2, 3]) == 2   # two uncolored (-1 == -1 is no clash
                                                 # on top: each is counted once)
    path = gg.from_nets(3, [[0, 1], [1, 2]])
    assert O.conflicts(path, [0, 0, 0]) == 3
    assert O.conflicts(path, [0, 1, 0]) == 0     # 0 and 2 share no net
    assert O.conflicts(path, [0, 0, 1]) == 2
    # a vertex clashing in two nets is counted once
    two = gg.from_nets(3, [[0, 1], [0, 2]])
    assert O.conflicts(two, [5, 5, 5]) == 3
    # a vertex without nets never clashes
    iso = gg.from_nets(3, [[0, 1]])
    assert O.conflicts(iso, [7, 8, 7]) == 0


def test_conflicts_against_incidence_matrix():
    rng = np.random.default_rng(31)
    for _ in range(60):
        n_a, n_b = int(rng.integers(1, 14)), int(rng.integers(1, 9))
        g, _ = random_tiny(rng, n_a, n_b, 5)
        M = conflict_matrix(g)
        c = rng.integers(-1, 4, size=n_a).astype(np.int32)
        same = (c[:, None] == c[None, :]) & M
        want = int(((c < 0) | same.any(axis=1)).sum())
        assert O.conflicts(g, c) == want


def test_max_nbor_hand_counts():
    # two vertices sharing two nets are one neighbour of each other
    g = gg.from_nets(2, [[0, 1], [0, 1]])
    best, sizes = O.max_nbor(g)
    assert best == 1 and sizes.tolist() == [1, 1]
    # one net of size s: s - 1 neighbours each
    for s in [1, 2, 9]:
        best, sizes = O.max_nbor(gg.from_nets(s, [list(range(s))]))
        assert best == s - 1 and sizes.tolist() == [s - 1] * s
    # overlapping nets {0,1,2}, {2,3}: vertex 2 sees 0, 1, 3 once each
    best, sizes = O.max_nbor(gg.from_nets(5, [[0, 1, 2], [2, 3]]))
    assert best == 3 and sizes.tolist() == [2, 2, 3, 1, 0]


@pytest.mark.parametrize("n", [5, 6, 9])
def test_max_nbor_stencil_closed_form(n):
    """9-point stencil: columns conflict iff |di| <= 2 and |dj| <= 2, so
    |nbor(i, j)| = (min(i,2) + min(n-1-i,2) + 1) (same for j) - 1: 24 inside,
    14 on an edge, 8 in a corner."""
    g = gg.stencil9(n)
    i, j = np.divmod(np.arange(n * n), n)
    span = lambda x: np.minimum(x, 2) + np.minimum(n - 1 - x, 2) + 1
    best, sizes = O.max_nbor(g)
    assert np.array_equal(sizes, span(i) * span(j) - 1)
    assert best == 24 and sizes[0] == 8 and sizes[2] == 14


def test_max_nbor_against_incidence_matrix():
    rng = np.random.default_rng(37)
    for _ in range(40):
        g, _ = random_tiny(rng, int(rng.integers(1, 16)), int(rng.integers(1, 10)), 6)
        best, sizes = O.max_nbor(g)
        want = conflict_matrix(g).sum(axis=1)
        assert np.array_equal(sizes, want) and best == int(want.max(initial=0))


def test_d2_conflicts_hand_counts():
    """Direct distance-2 check on a path 0-1-2-3 (Sec. II)."""
    ug = gg.from_edges(4, [(0, 1), (1, 2), (2, 3)])
    assert O.d2_conflicts(ug, [0, 1, 2, 0]) == 0   # 0 and 3 are at distance 3
    assert O.d2_conflicts(ug, [0, 1, 0, 2]) == 2   # 0 and 2 at distance 2
    assert O.d2_conflicts(ug, [0, 0, 1, 2]) == 2   # adjacent clash
    assert O.d2_conflicts(ug, [0, 1, -1, 0]) == 1  # uncolored
    assert O.d2_conflicts(ug, [0, 0, 0, 0]) == 4


# ------------------------------------------------------- net-based rounds
#
# Alg. 8 / Alg. 9 as the first round(s) of the N1-N2 / N2-N2 schedules of
# Sec. VI: every net reads the round's snapshot and proposes reverse
# first-fit colors to its uncolored members, every vertex keeps its owner
# net's proposal, a fixed vertex wins a clash.

def test_net_round_golden():
    fx = golden("rs_net_round.json")
    for key in ("path", "single_net"):
        case = fx[key]
        g = gg.from_nets(case["n_a"], case["nets"])
        r = O.rs_color(g, net_rounds=1)
        assert r.status == O.OK
        assert r.colors.tolist() == case["expected"]
        assert r.w_per_round.tolist() == case["w_per_round"]
        c_py, hist = rs_py.rs(case["n_a"], case["nets"], net_rounds=1)
        assert c_py == case["expected"] and hist == case["w_per_round"]
    st = fx["star_center_2"]
    cn = O.closed_nbhd(gg.from_edges(st["n"], st["edges"]))
    assert O.rs_color(cn, net_rounds=1, center_first=True).colors.tolist() == \
        st["expected_center_first"]
    assert O.rs_color(cn, net_rounds=1).colors.tolist() == st["expected_adjacency_order"]


def owner_nets(g):
    own = np.full(g.n_a, -1, np.int64)
    sizes = np.diff(g.b_ptr)
    for w in range(g.n_a):
        nets = g.a_idx[g.a_ptr[w]:g.a_ptr[w + 1]]
        if len(nets):
            own[w] = max(nets, key=lambda v: (sizes[v], v))
    return own


@pytest.mark.parametrize("center_first", [False, True])
def test_net_round_proposals_per_net(center_first):
    """Before its conflict removal, a net round gives the members that own a
    net distinct colors below |vtxs(v)| (the reverse first fit from
    |vtxs(v)| - 1 never reuses a color within a net and never goes below 0),
    and leaves exactly the vertices without nets uncolored."""
    rng = np.random.default_rng(41)
    for it in range(12):
        if center_first:
            ug = gg.rmat(7, 4, seed=60 + it)
            g = O.closed_nbhd(ug)
        else:
            g = gg.random_bipartite(300, 120, 3, seed=60 + it)
        r = O.rs_color(g, net_rounds=1, center_first=center_first, stop_after_waves=1,
                       stop_before_removal=True)
        assert r.status == O.STOPPED and r.wave == 1 and r.m == g.n_a
        own = owner_nets(g)
        c = r.colors
        assert np.array_equal(c < 0, own < 0)
        sizes = np.diff(g.b_ptr)
        for v in range(g.n_b):
            mem = g.b_idx[g.b_ptr[v]:g.b_ptr[v + 1]]
            owned = c[mem[own[mem] == v]]
            assert len(set(owned.tolist())) == len(owned)
            assert np.all((owned >= 0) & (owned < sizes[v]))


@pytest.mark.parametrize("net_rounds", [1, 2, 3])
def test_net_rounds_valid_and_match_python(net_rounds):
    """Colorings with net-based leading rounds are valid (Sec. II), every
    vertex-based round after them keeps the usual invariants, and the C
    oracle equals the independent Python statement, for all policies and
    ranks (the net round itself uses the reverse first fit whatever the
    policy)."""
    rng = np.random.default_rng(43 + net_rounds)
    for it in range(25):
        n_a, n_b = int(rng.integers(1, 40)), int(rng.integers(1, 25))
        g, nets = random_tiny(rng, n_a, n_b, 7)
        pol = POLICIES[it % 4]
        C, Q, T = int(rng.integers(1, 9)), int(rng.integers(1, 5)), int(rng.integers(0, 6))
        rank = rng.permutation(n_a).astype(np.int32) if it % 3 == 0 else None
        r = O.rs_color(g, pol, chunk=C, waves=Q, big_net=T, rank=rank, net_rounds=net_rounds)
        assert r.status == O.OK
        assert O.conflicts(g, r.colors) == 0
        c_py, hist = rs_py.rs(n_a, nets, pol, C, Q, T, None if rank is None else rank.tolist(),
                              net_rounds=net_rounds)
        assert r.colors.tolist() == c_py and r.w_per_round.tolist() == hist


def test_net_round_traversal_is_linear():
    """A net round reads every net touching W once: sum of |vtxs(v)| = nnz
    in the first round (every net has a member in W_0)."""
    g = gg.random_bipartite(500, 300, 4, seed=3)
    r = O.rs_color(g, net_rounds=1)
    sizes = np.diff(g.b_ptr)
    assert r.trav_per_round[0] == int(sizes[sizes > 0].sum()) == g.nnz
    r0 = O.rs_color(g)
    assert r0.trav_per_round[0] == int((sizes * (sizes - 1)).sum())


def test_net_round_d2gc_valid_by_distance():
    ug = gg.rmat(9, 8, seed=5)
    cn = O.closed_nbhd(ug)
    for pol in POLICIES:
        r = O.rs_color(cn, pol, chunk=8, waves=4, big_net=16, net_rounds=1, center_first=True)
        assert r.status == O.OK and O.d2_conflicts(ug, r.colors) == 0


# ------------------------------------------------------- smallest-last order

def sl_py(n_a, nets):
    """Smallest-last by its definition, with Python sets: remove a remaining
    vertex of smallest remaining conflict degree (ties: smallest id); the
    coloring order is the reverse removal order."""
    nb = [set() for _ in range(n_a)]
    for mem in nets:
        for u in mem:
            nb[u].update(x for x in mem if x != u)
    left, removal = set(range(n_a)), []
    while left:
        w = min(left, key=lambda x: (len(nb[x] & left), x))
        removal.append(w)
        left.remove(w)
    rank = [0] * n_a
    for pos, w in enumerate(reversed(removal)):
        rank[w] = pos
    return rank


def test_sl_hand_derived():
    """Path 0-1-2-3 (conflict graph): degrees 1,2,2,1, removal 0,1,2,3, so the
    coloring order is 3,2,1,0.  Star with center 0 and leaves 1,2,3: remove 1
    (degree 1), then 2; the center and 3 now both have degree 1, the smaller
    id (0) goes first, then 3: coloring order 3,0,2,1."""
    r, dg = O.sl_rank(gg.from_nets(4, [[0, 1], [1, 2], [2, 3]]))
    assert r.tolist() == [3, 2, 1, 0] and dg == 1
    r, dg = O.sl_rank(gg.from_nets(4, [[0, 1], [0, 2], [0, 3]]))
    assert r.tolist() == [1, 3, 2, 0] and dg == 1
    r, dg = O.sl_rank(gg.from_nets(5, [list(range(5))]))  # a clique: ids in order
    assert r.tolist() == [4, 3, 2, 1, 0] and dg == 4


def test_sl_matches_definition_and_degeneracy_bound():
    """Against the set-based statement on random tiny graphs; first fit in
    smallest-last order uses at most degeneracy + 1 colors (every vertex has
    at most `degeneracy` neighbours colored before it)."""
    rng = np.random.default_rng(51)
    for _ in range(40):
        n_a, n_b = int(rng.integers(1, 30)), int(rng.integers(1, 20))
        g, nets = random_tiny(rng, n_a, n_b, 6)
        r, dg = O.sl_rank(g)
        assert r.tolist() == sl_py(n_a, nets)
        assert sorted(r.tolist()) == list(range(n_a))
        c = O.seq_color(g, O.FF, rank=r)
        assert O.conflicts(g, c) == 0 and c.max() + 1 <= dg + 1
    g = gg.random_bipartite(400, 300, 4, seed=5)
    r, dg = O.sl_rank(g)
    assert O.seq_color(g, O.FF, rank=r).max() + 1 <= dg + 1
