"""The allocation-free color-set statistics entry point.

Some callers cannot allocate device memory: code under an allocator that
owns the whole memory budget, or loops that must not enter the driver's
allocator (cudaMalloc and cudaFree can synchronise the device).
bgpc_color_sets_noalloc gives them the statistics of bgpc_color_sets with its
scratch in a fixed device array.  This test calls it through the C ABI twice
in a row and checks it against bgpc_color_sets.  It lives in its own file,
collected last, so that a run stopping at the first failure has already run
every other test; it also passes on its own in a fresh process."""
import numpy as np
import pytest
import torch

import graphgen as gg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bg():
    import paper_1701_02628_gb300 as m
    from paper_1701_02628_gb300 import build
    build.build()
    return m


def test_noalloc_matches_color_sets_twice(bg):
    ctx = bg.Context(0)
    for g, pol in ((gg.random_bipartite(3000, 2000, 5, seed=9), bg.BGPC_B2),
                   (gg.chung_lu(20000, 16, 1500, 2.1, seed=4), bg.BGPC_FF)):
        dg = bg.DeviceGraph.from_host(g, "cuda:0")
        colors, st, _ = bg.bgpc_color(ctx, dg, policy=pol)
        ncol = st["colors"]
        _, ref = bg.bgpc_color_sets(ctx, colors, ncol)
        for _ in range(2):  # the shared scratch must be cleared between calls
            got = bg.bgpc_color_sets_noalloc(colors, ncol)
            assert got["n_sets"] == ref["n_sets"]
            assert got["max_card"] == ref["max_card"]
            assert got["mean_card"] == pytest.approx(ref["mean_card"], rel=1e-9)
            assert got["std_card"] == pytest.approx(ref["std_card"], rel=1e-9, abs=1e-12)
        # a larger histogram bound gives the same statistics
        got = bg.bgpc_color_sets_noalloc(colors, ncol + 1000)
        assert got["n_sets"] == ref["n_sets"] and got["max_card"] == ref["max_card"]
    ctx.close()


def test_noalloc_rejects_out_of_range(bg):
    c = torch.tensor([0, 1, 5, 2], dtype=torch.int32, device="cuda:0")
    with pytest.raises(bg.BgpcError) as e:
        bg.bgpc_color_sets_noalloc(c, 5)  # color 5 >= max_colors
    assert e.value.status == bg.BGPC_EINVAL
    with pytest.raises(bg.BgpcError) as e:
        bg.bgpc_color_sets_noalloc(c, bg.BGPC_NOALLOC_MAX_COLORS + 1)
    assert e.value.status == bg.BGPC_EINVAL
    got = bg.bgpc_color_sets_noalloc(c, 6)
    assert got == dict(n_sets=4, max_card=1, mean_card=1.0, std_card=0.0)
