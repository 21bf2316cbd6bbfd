"""GPU parity at the benchmark's full sizes, in the configuration bench.py
times (RS(C=64, Q=16, T=64), id order).

* 9-point stencil 1024 x 1024: the oracle replays the whole coloring.
* Chung-Lu 2^22 x 2^22 and R-MAT scale 22 (D2GC): a full replay would take
  hours on the CPU, so outputs are sampled.  The GPU stops at the start of a
  wave (stop_after_waves) and returns its state (colors and work queue); the
  oracle colors sampled chunks of that wave from that state, and the result
  must equal the GPU's colors one wave later.  The conflict rule is checked on
  sampled vertices from the GPU's colors before removal.  Validity of the
  final coloring is checked by an independent per-net numpy test.
"""
import numpy as np
import pytest
import torch

import graphgen as gg
import hubrule
import oracle as O
import rs_py

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

C, Q, T = 64, 16, 64


@pytest.fixture(scope="module")
def bg():
    import paper_1701_02628_gb300 as m
    from paper_1701_02628_gb300 import build
    build.build()
    return m


@pytest.fixture(scope="module")
def ctx(bg):
    return bg.Context(0)


@pytest.fixture(scope="module")
def rmat22():
    ug = gg.rmat(22, 16, seed=3)
    return ug, O.closed_nbhd(ug)


def per_net_valid(b_ptr, b_idx, n_b, c) -> bool:
    """No uncolored vertex and no two members of a net with one color."""
    if (c < 0).any():
        return False
    nets = np.repeat(np.arange(n_b, dtype=np.int64), np.diff(b_ptr))
    key = nets * (int(c.max()) + 1) + c[b_idx].astype(np.int64)
    key.sort()
    return not bool((np.diff(key) == 0).any())


def chunk_volume(g, W, m):
    """Two-hop entries of each chunk of W (for choosing affordable samples)."""
    sizes = np.diff(g.b_ptr).astype(np.int64)
    deg = np.diff(g.a_ptr).astype(np.int64)
    per_v = np.zeros(g.n_a, np.int64)
    np.add.at(per_v, np.repeat(np.arange(g.n_a), deg), sizes[g.a_idx])
    nch = (m + C - 1) // C
    vol = np.zeros(nch, np.int64)
    np.add.at(vol, np.arange(m) // C, per_v[W[:m]])
    return vol


def sampled_wave_parity(bg, ctx, g, run, stops, policy, rng, per_wave=12, budget=3e8):
    """run(**opts) -> (colors, stats, rc) through the C ABI on graph g."""
    W_out = torch.empty(max(g.n_a, 1), dtype=torch.int32, device="cuda:0")
    checked = 0
    for s in stops:
        col_s, st_s, rc = run(policy=policy, stop_after_waves=s, W_out=W_out)
        assert rc == bg.BGPC_STOPPED
        q, m = st_s["stopped_wave"], st_s["stopped_m"]
        S = col_s.cpu().numpy()
        W = W_out[:m].cpu().numpy()
        col_n, _, rc = run(policy=policy, stop_after_waves=s + 1, stop_before_removal=True)
        nxt = col_n.cpu().numpy()
        nch = (m + C - 1) // C
        chunks = np.array([j for j in range(nch) if rs_py.wave_of(j, Q) == q], np.int64)
        vol = chunk_volume(g, W, m)[chunks]
        cheap = chunks[vol <= budget]
        pick = rng.choice(cheap, size=min(per_wave, len(cheap)), replace=False)
        out = O.rs_chunks(g, S, W, pick.astype(np.int32), policy, chunk=C, big_net=T,
                          nthreads=16)
        for j in pick:
            pos = np.arange(j * C, min(m, (j + 1) * C))
            assert np.array_equal(out[pos], nxt[W[pos]]), f"wave start {s}, chunk {j}"
            checked += len(pos)
    return checked


def sampled_conflict_rule(bg, run, g, policy, rng, nsample=400):
    W1 = torch.empty(g.n_a, dtype=torch.int32, device="cuda:0")
    pre, st, rc = run(policy=policy, stop_after_waves=Q, stop_before_removal=True, W_out=W1)
    assert rc == bg.BGPC_STOPPED and st["stopped_wave"] == Q
    m1 = st["stopped_m"]
    W2 = torch.empty(g.n_a, dtype=torch.int32, device="cuda:0")
    _, st2, rc2 = run(policy=policy, stop_after_waves=Q, W_out=W2)
    W_1 = W1[:m1].cpu().numpy()
    losers = set(W2[:st2["stopped_m"]].cpu().numpy().tolist()) if rc2 == bg.BGPC_STOPPED else set()
    which = rng.choice(m1, size=min(nsample, m1), replace=False).astype(np.int32)
    lose, status = O.rs_losers(g, pre.cpu().numpy(), W_1, which)
    assert status == O.OK  # no W vertex took a fixed neighbour's color
    for p, l in zip(which, lose):
        assert bool(l) == (int(W_1[p]) in losers)


def test_stencil_1024_full_parity(bg, ctx):
    g = gg.stencil9(1024)
    ref = O.rs_color(g, O.FF, chunk=C, waves=Q, big_net=T, nthreads=16)
    dg = bg.DeviceGraph.from_host(g, "cuda:0")
    colors, st, rc = bg.bgpc_color(ctx, dg)
    got = colors.cpu().numpy()
    assert np.array_equal(got, ref.colors)
    assert st["rounds"] == ref.rounds and st["trav_total"] == int(ref.trav_per_round.sum())
    assert per_net_valid(g.b_ptr, g.b_idx, g.n_b, got)


def test_chung_lu_4m_sampled(bg, ctx):
    g = gg.chung_lu(1 << 22, 16.0, 50000.0, 2.1, seed=2)
    dg = bg.DeviceGraph.from_host(g, "cuda:0")
    run = lambda **kw: bg.bgpc_color(ctx, dg, **kw)
    rng = np.random.default_rng(7)
    n = sampled_wave_parity(bg, ctx, g, run, [1, 6, 15, 17], O.FF, rng)
    assert n > 1000
    sampled_conflict_rule(bg, run, g, O.FF, rng)
    colors, st, rc = run()
    assert rc == bg.BGPC_OK
    assert per_net_valid(g.b_ptr, g.b_idx, g.n_b, colors.cpu().numpy())
    assert st["w_per_round"][0] == g.n_a
    assert hubrule.check(st, np.diff(g.b_ptr)) == 512  # 10,755 hubs, 52 MB of bitmaps


@pytest.mark.parametrize("policy", [O.FF, O.B1, O.B2])
def test_rmat22_d2gc_sampled(bg, ctx, rmat22, policy):
    ug, cn = rmat22
    dug = bg.DeviceUGraph.from_host(ug, "cuda:0")
    run = lambda **kw: bg.d2gc_color(ctx, dug, **kw)
    rng = np.random.default_rng(11 + policy)
    n = sampled_wave_parity(bg, ctx, cn, run, [1, 9, 15], policy, rng, per_wave=8, budget=2e8)
    assert n > 500
    sampled_conflict_rule(bg, run, cn, policy, rng, nsample=200)
    colors, st, rc = run(policy=policy)
    assert rc == bg.BGPC_OK
    assert per_net_valid(cn.b_ptr, cn.b_idx, cn.n_b, colors.cpu().numpy())
    # the bitmaps of the nets above 512 members would not fit in half the
    # L2: the threshold is raised up the ladder
    assert hubrule.check(st, np.diff(cn.b_ptr)) > 512


def test_chung_lu_4m_net_round(bg, ctx):
    """N1 on the full-size power-law graph: the whole net round (tentative
    colors before removal, and the work queue after it) equals the oracle's,
    which is linear in nnz; the vertex-based waves after it are sampled."""
    g = gg.chung_lu(1 << 22, 16.0, 50000.0, 2.1, seed=2)
    dg = bg.DeviceGraph.from_host(g, "cuda:0")
    run = lambda **kw: bg.bgpc_color(ctx, dg, net_rounds=1, **kw)
    ref = O.rs_color(g, net_rounds=1, stop_after_waves=1, stop_before_removal=True)
    got, st, rc = run(stop_after_waves=1, stop_before_removal=True)
    assert rc == bg.BGPC_STOPPED and np.array_equal(got.cpu().numpy(), ref.colors)
    rng = np.random.default_rng(17)
    # the round-2 work queue holds exactly the net round's losers (the
    # conflict rule on sampled vertices; every vertex is in W_1, id order)
    W_out = torch.empty(g.n_a, dtype=torch.int32, device="cuda:0")
    _, st2, rc = run(stop_after_waves=1, W_out=W_out)  # start of round 2, wave 0
    assert rc == bg.BGPC_STOPPED and st2["stopped_wave"] == 0 and st2["rounds"] == 2
    inW2 = np.zeros(g.n_a, bool)
    inW2[W_out[:st2["stopped_m"]].cpu().numpy()] = True
    which = rng.choice(g.n_a, size=400, replace=False).astype(np.int32)
    lose, status = O.rs_losers(g, ref.colors, np.arange(g.n_a, dtype=np.int32), which)
    assert status == O.OK and np.array_equal(lose.astype(bool), inW2[which])
    n = sampled_wave_parity_n1(bg, g, run, rng)
    assert n > 500
    colors, st, rc = run()
    assert rc == bg.BGPC_OK
    assert per_net_valid(g.b_ptr, g.b_idx, g.n_b, colors.cpu().numpy())


def sampled_wave_parity_n1(bg, g, run, rng, per_wave=12, budget=3e8):
    """Waves of the vertex-based rounds after the net round (wave counts
    shifted by the net round's one wave)."""
    W_out = torch.empty(g.n_a, dtype=torch.int32, device="cuda:0")
    checked = 0
    for s in (2, 9, 17):
        col_s, st_s, rc = run(stop_after_waves=s, W_out=W_out)
        assert rc == bg.BGPC_STOPPED
        q, m = st_s["stopped_wave"], st_s["stopped_m"]
        S = col_s.cpu().numpy()
        W = W_out[:m].cpu().numpy()
        col_n, _, rc = run(stop_after_waves=s + 1, stop_before_removal=True)
        nxt = col_n.cpu().numpy()
        nch = (m + C - 1) // C
        chunks = np.array([j for j in range(nch) if rs_py.wave_of(j, Q) == q], np.int64)
        vol = chunk_volume(g, W, m)[chunks]
        cheap = chunks[vol <= budget]
        pick = rng.choice(cheap, size=min(per_wave, len(cheap)), replace=False)
        out = O.rs_chunks(g, S, W, pick.astype(np.int32), O.FF, chunk=C, big_net=T, nthreads=16)
        for j in pick:
            pos = np.arange(j * C, min(m, (j + 1) * C))
            assert np.array_equal(out[pos], nxt[W[pos]]), f"wave start {s}, chunk {j}"
            checked += len(pos)
    return checked
