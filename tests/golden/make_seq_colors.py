"""Writes seq_colors_fullsize.json: the sequential greedy coloring (the
oracle's O-1, i.e. the paper's sequential V-V of Table II, one thread, no
conflicts) of the full-size benchmark graphs, under first fit and the two
balancing heuristics of Sec. V, with the color-set statistics of Table VI.

These are the "plain method" numbers the benchmark puts beside the
round-synchronous GPU colorings.  O-1 is Theta(E2) on one thread (minutes
per graph), too slow for every benchmark run, so it is run once by this
script, which calls only the oracle and the generators.  Each record carries
a SHA-1 of the graph's arrays: the Chung-Lu generator uses libm pow, so a
graph built on another platform may differ, and then the record does not
apply to it.

Usage: python tests/golden/make_seq_colors.py [graph ...]
(graphs: stencil, chunglu22, rmat22; default all; one process per graph and
policy, run in parallel)."""
import concurrent.futures as cf
import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "seq_colors_fullsize.json")


def graph_sha1(g) -> str:
    h = hashlib.sha1()
    for a in (g.a_ptr, g.a_idx, g.b_ptr, g.b_idx):
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def make(name):
    import graphgen as gg
    import oracle as O
    if name == "stencil":
        return gg.stencil9(1024)
    if name == "chunglu22":
        return gg.chung_lu(1 << 22, 16.0, 50000.0, 2.1, seed=2)
    if name == "rmat22":
        ug = gg.rmat(22, 16, seed=3)
        g = O.closed_nbhd(ug)
        g.name = ug.name + "_closed"
        return g
    raise ValueError(name)


def one(name, policy):
    import oracle as O
    g = make(name)
    t0 = time.time()
    c = O.seq_color(g, policy)
    secs = time.time() - t0
    b = O.balance(c)
    return {"graph": name, "graph_name": getattr(g, "name", name), "sha1": graph_sha1(g),
            "policy": {O.FF: "FF", O.B1: "B1", O.B2: "B2"}[policy],
            "colors": int(c.max()) + 1, "n_sets": b["colors"], "max_card": b["max_card"],
            "mean_card": b["mean_card"], "std_card": b["std_card"], "seconds": secs}


def main():
    import oracle as O
    O.build()
    names = sys.argv[1:] or ["stencil", "chunglu22", "rmat22"]
    jobs = [(n, p) for n in names for p in (O.FF, O.B1, O.B2)]
    old = json.load(open(OUT)) if os.path.exists(OUT) else []
    keep = [r for r in old if r["graph"] not in names]
    ctx = __import__("multiprocessing").get_context("spawn")
    with cf.ProcessPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 1),
                                mp_context=ctx) as ex:
        recs = list(ex.map(one, *zip(*jobs)))
    with open(OUT, "w") as f:
        json.dump(keep + recs, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
