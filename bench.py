#!/usr/bin/env python
"""Benchmark of the GB300 BGPC path on the Jacobian-like workload.

One step = one complete coloring (setup, every round of coloring waves,
publication, conflict detection and compaction) of each graph of the
workload, through the C ABI, with the graphs already resident in HBM:

  * 9-point stencil Jacobian, 1024 x 1024 (1,048,576 nets and columns),
  * Chung-Lu power-law bipartite graph, 2^22 x 2^22, mean degree 16,
    weights up to 50,000, exponent 2.1,

plain first-fit round-synchronous coloring RS(C=64, Q=16, T=64), id order.
The metric is traversed two-hop entries per second: sum over the rounds of
sum over W_r of sum over nets(w) of (|vtxs(v)| - 1) (one full sweep of the
vertex-based gather is E2 = sum_v |vtxs(v)| (|vtxs(v)| - 1)), divided by the
device time of the step.  Inputs (1.3 GB of graph and mirrors per step) are
larger than the 129 MB L2, so no flush is needed between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Multi-GPU (torchrun): every rank colors its own replica (the single-graph
path does not shard); value = all ranks' entries / max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "2-hop edges colored/s vs HBM roofline; colors used & balance vs plain/oracle"
UNIT = "2-hop entries/s"
WORKLOAD = ("BGPC Jacobian-like: stencil9 1024x1024 + Chung-Lu 2^22x2^22 (mean 16, max 50k, "
            "exp 2.1); plain first fit RS(C=64,Q=16,T=64), id order")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


WORKLOADS = {
    # the benchmark workload: both Jacobian-like graphs of the BGPC configuration
    "jacobian": WORKLOAD,
    # smaller cases for profiler captures (same generators, fewer vertices)
    "chunglu20": "Chung-Lu 2^20x2^20 (mean 16, max 12.5k, exp 2.1), RS(64,16,64) first fit",
    "chunglu22": "Chung-Lu 2^22x2^22 (mean 16, max 50k, exp 2.1), RS(64,16,64) first fit",
    "stencil": "stencil9 1024x1024, RS(64,16,64) first fit",
    "rmat22": "D2GC on R-MAT scale 22 (edge factor 16, a=.57 b=.19 c=.19), RS(64,16,64) first fit",
    # the batched configuration: 512 independent graphs, one bgpc_color_batched call
    "batch512": ("512 graphs, |V_A| log-uniform [1e3,1e6], |V_B| = |V_A|*U[0.5,2], degree "
                 "Poisson(8) clipped to [1,64]; RS(64,16,64) first fit, id order, one batched call"),
    # the first 128 graphs of the same batch, for profiler captures
    "batch128": ("128 graphs of the batched workload (the first 128 of batch512), one batched "
                 "call"),
}


def make_workload(name="jacobian"):
    import graphgen as gg
    if name == "chunglu20":
        return [gg.chung_lu(1 << 20, 16.0, 12500.0, 2.1, seed=2)]
    if name == "stencil":
        return [gg.stencil9(1024)]
    if name == "chunglu22":
        return [gg.chung_lu(1 << 22, 16.0, 50000.0, 2.1, seed=2)]
    if name == "batch512":
        return [gg.batch_graph(17, i) for i in range(512)]
    if name == "batch128":
        return [gg.batch_graph(17, i) for i in range(128)]
    if name == "rmat22":
        return [gg.rmat(22, 16, seed=3)]
    return [gg.stencil9(1024), gg.chung_lu(1 << 22, 16.0, 50000.0, 2.1, seed=2)]


def e2_of(g) -> int:
    """E2 = sum over nets of |vtxs(v)| (|vtxs(v)| - 1): one full sweep of the
    vertex-based gather (Sec. III); for an undirected graph (D2GC) the nets
    are the closed neighbourhoods, |N[v]| = deg(v) + 1."""
    if hasattr(g, "b_ptr"):
        s = np.diff(g.b_ptr).astype(np.int64)
    else:
        s = np.diff(g.ptr).astype(np.int64) + 1
    return int((s * (s - 1)).sum())


def graph_sha1(g) -> str:
    import hashlib
    h = hashlib.sha1()
    arrs = (g.a_ptr, g.a_idx, g.b_ptr, g.b_idx) if hasattr(g, "b_ptr") else (g.ptr, g.idx)
    for a in arrs:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def closed_sha1(ug) -> str:
    """SHA-1 of the closed-neighbourhood CSR of an undirected graph (N[u] =
    {u} u adj(u), sorted: the a_ptr/a_idx = b_ptr/b_idx of D2GC's bipartite
    form), built with numpy, to match the stored sequential-greedy records."""
    import hashlib
    n = ug.n
    ptr = ug.ptr.astype(np.int64)
    deg = np.diff(ptr)
    rows = np.repeat(np.arange(n, dtype=np.int64), deg)
    below = ug.idx.astype(np.int64) < rows          # neighbours before u in N[u]
    nbelow = np.bincount(rows[below], minlength=n)
    cidx = np.empty(ptr[-1] + n, np.int32)
    cidx[np.arange(ptr[-1]) + rows + (~below)] = ug.idx
    cidx[ptr[:-1] + np.arange(n) + nbelow] = np.arange(n, dtype=np.int32)
    cptr = (ptr + np.arange(n + 1)).astype(np.int32)
    h = hashlib.sha1()
    for a in (cptr, cidx, cptr, cidx):
        h.update(a.tobytes())
    return h.hexdigest()


def seq_records():
    """Sequential greedy (the oracle's O-1, the paper's sequential V-V)
    colorings of the full-size graphs, stored by tests/golden/make_seq_colors.py
    (O-1 is minutes per graph on one core, too slow for every run)."""
    p = os.path.join(ROOT, "tests", "golden", "seq_colors_fullsize.json")
    if not os.path.exists(p):
        return []
    with open(p) as f:
        return json.load(f)


def seq_for(records, sha1, policy):
    for r in records:
        if r["sha1"] == sha1 and r["policy"] == policy:
            return {k: r[k] for k in ("colors", "n_sets", "max_card", "mean_card", "std_card")}
    return None


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def kernel_traffic(kernel: str, bytes_per_launch: float):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, scaled from the captured launches' algorithmic bytes to this
    run's mean launch (traffic grows with the entries streamed); None when
    the kernel's source changed after the capture."""
    import hashlib
    p = os.path.join(ROOT, "profiles", f"traffic_{kernel}.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        rec = json.load(f)
    src = os.path.join(ROOT, "paper_1701_02628_gb300", "csrc", rec["source"])
    with open(src, "rb") as f:
        if hashlib.sha1(f.read()).hexdigest() != rec["source_sha1"]:
            return None
    return rec["dram_bytes"] / rec["algorithmic_bytes"] * bytes_per_launch


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, x: float, device) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------- CPU leg

def oracle_sample(graphs, budget_s: float, nthreads: int):
    """Time the CPU oracle, as it stands, on a bounded sample of the workload:
    the full round-synchronous replay of the stencil graph, plus round-1
    chunks of the power-law graph evenly spread over its work queue (snapshot:
    nothing colored yet), as many as fit the time budget.  The two graphs'
    rates are also reported separately (the mix depends on the budget)."""
    import oracle as O
    stencil, cl = graphs
    t0 = time.perf_counter()
    r = O.rs_color(stencil, O.FF, nthreads=nthreads)
    t_st = time.perf_counter() - t0
    e_st = int(r.trav_per_round.sum())
    entries = e_st
    spent = t_st
    W = np.arange(cl.n_a, dtype=np.int32)
    S = np.full(cl.n_a, -1, np.int32)
    nch = (cl.n_a + 63) // 64
    deg = np.diff(cl.a_ptr).astype(np.int64)
    sizes = np.diff(cl.b_ptr).astype(np.int64)
    per_vertex = np.zeros(cl.n_a, np.int64)
    np.add.at(per_vertex, np.repeat(np.arange(cl.n_a), deg), sizes[cl.a_idx] - 1)
    chunks_done = 0
    batch = max(nthreads, 8)
    stride = 97
    order = (np.arange(nch, dtype=np.int64) * stride) % nch
    e_cl, t_cl = 0, 0.0
    while spent < budget_s and chunks_done < nch:
        ch = order[chunks_done:chunks_done + batch].astype(np.int32)
        t1 = time.perf_counter()
        O.rs_chunks(cl, S, W, ch, O.FF, chunk=64, big_net=64, nthreads=nthreads)
        dt = time.perf_counter() - t1
        spent += dt
        t_cl += dt
        for j in ch:
            e_cl += int(per_vertex[j * 64:(j + 1) * 64].sum())
        chunks_done += len(ch)
    entries += e_cl
    return {"value": entries / spent, "unit": UNIT, "cores": nthreads, "kind": "oracle",
            "sample": (f"full RS replay of stencil9 1024x1024 ({e_st} "
                       f"entries, {r.rounds} rounds) + {chunks_done} of {nch} round-1 chunks of "
                       f"the Chung-Lu graph ({nthreads} threads, {spent:.1f} s)"),
            "per_graph": {"stencil9_1024x1024": {"entries_per_s": e_st / t_st, "seconds": t_st},
                          "chung_lu_2^22_round1_chunks": {
                              "entries_per_s": e_cl / t_cl if t_cl > 0 else None,
                              "chunks": chunks_done, "seconds": t_cl}},
            "cpu_model": cpu_model(),
            "seconds": spent, "entries": entries}


def run_reference(args):
    world, rank, local = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0
    if rank != 0:
        return
    import oracle
    oracle.build()
    graphs = make_workload()
    nthreads = os.cpu_count() or 1
    per_step = max(3.0, 60.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        oracle_sample(graphs, per_step, nthreads)
    vals, secs = [], []
    for _ in range(args.steps):
        s = oracle_sample(graphs, per_step, nthreads)
        vals.append(s["entries"])
        secs.append(s["seconds"])
    value = sum(vals) / sum(secs)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * sum(secs) / len(secs), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nthreads, "kind": "oracle",
                             "sample": s["sample"], "per_graph": s["per_graph"],
                             "cpu_model": s["cpu_model"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- GPU leg

def learned_order_report(bg, ctx, dev, chung_lu_dg):
    """The learned vertex order (features -> MLP -> rank) against id order:
    trained on 16 graphs of the batched workload (seed 23), evaluated on the
    Chung-Lu 2^22 graph and on 64 fresh graphs of the batched workload
    (seed 29, |V_A| log-uniform in [1e3, 1e6]).  Reports colors used, the
    color-set balance and the end-to-end time (order + coloring) against the
    coloring in id order."""
    import torch
    import graphgen as gg
    train = [bg.DeviceGraph.from_host(gg.batch_graph(23, i, lo=1e3, hi=1e5), dev)
             for i in range(16)]
    t0 = time.time()
    mlp, losses = bg.train_order(ctx, train, torch.from_numpy(gg.mlp_init(7)).to(dev),
                                 steps=300, lr=3e-3)
    torch.cuda.synchronize()
    t_train = time.time() - t0
    stream = torch.cuda.current_stream()

    def timed(fn, reps=3):
        fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1) / reps

    def id_run(dg):
        return bg.bgpc_color(ctx, dg, want_balance=True)[1]

    def learned_run(dg):
        return bg.bgpc_color(ctx, dg, rank=bg.learned_rank(ctx, dg, mlp), want_balance=True)[1]

    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record()
    bg.learned_rank(ctx, chung_lu_dg, mlp)
    s1.record()
    torch.cuda.synchronize()
    st_id, ms_id = timed(lambda: id_run(chung_lu_dg))
    st_l, ms_l = timed(lambda: learned_run(chung_lu_dg))
    bal = lambda st: {k: st[k] for k in ("n_sets", "max_card", "mean_card", "std_card")}
    cl = {"colors_id": st_id["colors"], "colors_learned": st_l["colors"],
          "ms_order": s0.elapsed_time(s1), "ms_id_order_coloring": ms_id,
          "ms_learned_order_and_coloring": ms_l, "rounds_id": st_id["rounds"],
          "rounds_learned": st_l["rounds"], "balance_id": bal(st_id),
          "balance_learned": bal(st_l)}
    fresh_id, fresh_l, std_id, std_l, t_id, t_l = [], [], [], [], 0.0, 0.0
    for i in range(64):
        dg = bg.DeviceGraph.from_host(gg.batch_graph(29, i), dev)
        a, ta = timed(lambda: id_run(dg), reps=1)
        b, tb = timed(lambda: learned_run(dg), reps=1)
        fresh_id.append(a["colors"])
        fresh_l.append(b["colors"])
        std_id.append(a["std_card"] / a["mean_card"])
        std_l.append(b["std_card"] / b["mean_card"])
        t_id += ta
        t_l += tb
    # the three orders side by side on 16 fresh graphs (|V_A| up to 1e5: the
    # smallest-last order is built by one host thread)
    cmp_n, cmp_sl, cmp_l, t_sl = [], [], [], 0.0
    for i in range(16):
        dg = bg.DeviceGraph.from_host(gg.batch_graph(29, 100 + i, lo=1e3, hi=1e5), dev)
        cmp_n.append(id_run(dg)["colors"])
        t0 = time.time()
        srank, _ = bg.sl_rank(ctx, dg)
        t_sl += time.time() - t0
        cmp_sl.append(bg.bgpc_color(ctx, dg, rank=srank)[1]["colors"])
        cmp_l.append(learned_run(dg)["colors"])
    orders = {"graphs": 16, "colors_natural_mean": float(np.mean(cmp_n)),
              "colors_smallest_last_mean": float(np.mean(cmp_sl)),
              "colors_learned_mean": float(np.mean(cmp_l)),
              "smallest_last_fewer_than_natural": int(sum(a < b for a, b in zip(cmp_sl, cmp_n))),
              "learned_fewer_than_natural": int(sum(a < b for a, b in zip(cmp_l, cmp_n))),
              "smallest_last_host_seconds": t_sl}
    return {"model": "MLP 8-64-64-1, bf16 weights, fp32 arithmetic, Adam",
            "orders_compared": orders,
            "train": {"graphs": 16, "steps": len(losses), "loss_first": losses[0],
                      "loss_last": losses[-1], "seconds": t_train},
            "chung_lu_2^22": cl,
            "fresh_batch_graphs": {"graphs": 64, "colors_id_mean": float(np.mean(fresh_id)),
                                   "colors_learned_mean": float(np.mean(fresh_l)),
                                   "fewer_colors": int(sum(a > b for a, b in zip(fresh_id, fresh_l))),
                                   "more_colors": int(sum(a < b for a, b in zip(fresh_id, fresh_l))),
                                   "card_cv_id_mean": float(np.mean(std_id)),
                                   "card_cv_learned_mean": float(np.mean(std_l)),
                                   "ms_id_total": t_id, "ms_learned_total": t_l}}


def d2gc_report(bg, ctx, dev, steps: int, warmup: int, records):
    """D2GC on R-MAT scale 22 (the distance-2 configuration) under first fit
    and both balancing heuristics of Sec. V, with Table VI's color-set
    statistics, against the sequential greedy coloring of the same graph.
    Timed with CUDA events on the launch stream, graph resident in HBM."""
    import torch
    import graphgen as gg
    ug = gg.rmat(22, 16, seed=3)
    dug = bg.DeviceUGraph.from_host(ug, dev)
    colors = torch.empty(ug.n, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    e2 = e2_of(ug)
    sha = closed_sha1(ug)
    deg = np.diff(ug.ptr)
    out = {"graph": ug.name, "n": int(ug.n), "adjacency_entries": int(ug.nnz), "E2": e2,
           "max_closed_nbhd": int(deg.max()) + 1, "policies": {}}
    for pol, name in ((bg.BGPC_FF, "FF"), (bg.BGPC_B1, "B1"), (bg.BGPC_B2, "B2")):
        for _ in range(warmup):
            bg.d2gc_color(ctx, dug, colors, policy=pol, want_balance=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            _, st, _ = bg.d2gc_color(ctx, dug, colors, policy=pol, want_balance=True)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        seq = seq_for(records, sha, name)
        rec = {"ms": ms, "rounds": st["rounds"], "colors": st["colors"], "n_sets": st["n_sets"],
               "max_card": st["max_card"], "mean_card": st["mean_card"],
               "std_card": st["std_card"], "trav_total": st["trav_total"],
               "entries_per_s": st["trav_total"] / (ms / 1000.0),
               "E2_per_s": e2 / (ms / 1000.0),
               "colors_seq": seq["colors"] if seq else None,
               "colors_vs_seq": st["colors"] / seq["colors"] if seq else None,
               "seq_balance": seq}
        out["policies"][name] = rec
    out["schedules"] = schedule_report(bg, ctx, [dug], [ug], steps, records, d2=True)[0]
    ff = out["policies"]["FF"]
    for name in ("B1", "B2"):
        r = out["policies"][name]
        r["vs_FF"] = {"colors": r["n_sets"] / ff["n_sets"], "mean_card": r["mean_card"] / ff["mean_card"],
                      "std_card": r["std_card"] / ff["std_card"] if ff["std_card"] else None,
                      "time": r["ms"] / ff["ms"]}
    return out


def schedule_report(bg, ctx, dgs, graphs, steps: int, records, d2=False):
    """The schedules of Sec. VI side by side on the same graphs: V-* (every
    round vertex-based, the timed configuration) and N1-* (the first round
    net-based, Alg. 8 / Alg. 9), each a complete coloring timed with CUDA
    events: time, rounds, colors, traversal over E2 and E2 per second."""
    import torch
    stream = torch.cuda.current_stream()
    out = []
    for g, dg in zip(graphs, dgs):
        e2 = e2_of(g)
        rec = {"graph": g.name}
        for name, nr in (("V", 0), ("N1", 1)):
            fn = (lambda: bg.d2gc_color(ctx, dg, net_rounds=nr)) if d2 else \
                 (lambda: bg.bgpc_color(ctx, dg, net_rounds=nr))
            fn()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(steps):
                _, st, _ = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            rec[name] = {"ms": ms, "rounds": st["rounds"], "colors": st["colors"],
                         "w_per_round": st["w_per_round"][:8],
                         "trav_over_E2": st["trav_total"] / e2, "E2_per_s": e2 / (ms / 1000.0)}
        out.append(rec)
    return out


def run_gpu(args):
    import torch
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    from paper_1701_02628_gb300 import build as cbuild
    if rank == 0 or not cbuild.up_to_date():
        cbuild.build()
    barrier(world)
    import paper_1701_02628_gb300 as bg

    graphs = make_workload(args.workload)
    d2 = args.workload == "rmat22"
    ctx = bg.Context(local)
    if d2:
        dgs = [bg.DeviceUGraph.from_host(g, dev) for g in graphs]
        n_of = lambda g: g.n
    else:
        dgs = [bg.DeviceGraph.from_host(g, dev) for g in graphs]
        n_of = lambda g: g.n_a
    colors = [torch.empty(n_of(g), dtype=torch.int32, device=dev) for g in graphs]
    stream = torch.cuda.current_stream()

    batched = args.workload.startswith("batch")

    last_rounds = []

    def step(profile=False):
        if batched:
            _, st, rounds, _ = bg.bgpc_color_batched(ctx, dgs, colors, profile=profile)
            last_rounds[:] = rounds
            return [st]
        sts = []
        for dg, c in zip(dgs, colors):
            if d2:
                _, st, _ = bg.d2gc_color(ctx, dg, c, profile=profile)
            else:
                _, st, _ = bg.bgpc_color(ctx, dg, c, profile=profile)
            sts.append(st)
        return sts

    for _ in range(args.warmup):
        step()
    # correctness of the timed configuration: valid colorings
    if not d2:
        for dg, c in zip(dgs, colors):
            assert bg.bgpc_validate(ctx, dg, c) == 0, "invalid coloring"

    sampler = ClockSampler(local) if rank == 0 else None
    barrier(world)
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
        time.sleep(0.4)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    all_stats = []
    for _ in range(args.steps):
        all_stats.append(step(profile=True))
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop() if sampler else None
    ms = ev0.elapsed_time(ev1)
    ms_max = max_over_ranks(world, ms, dev)
    ms_step = ms_max / args.steps

    entries_step = sum(st["trav_total"] for st in all_stats[-1])
    value = world * entries_step * args.steps / (ms_max / 1000.0)
    launches = sum(st["kernel_launches"] for sts in all_stats for st in sts)
    e2_step = sum(e2_of(g) for g in graphs)
    hub_step = sum(st["trav_hub"] for st in all_stats[-1])

    # roofline of the dominant kernel: algorithmic bytes per launch / mean
    # launch duration, both over the timed region.  The gather kernel streams
    # the mirror entries of the large vertices' nets except the hub nets
    # (4 B per entry), reads a hub net's color bitmap instead (4 B per word),
    # plus 12 B per incidence (a_idx and the b_ptr pair); the resolve kernel
    # streams the small vertices' entries, plus 28 B per small vertex.
    def tot(key):
        return sum(st[key] for sts in all_stats for st in sts)
    n_launch = tot("color_launches")
    kern = {
        "k_gather": (tot("ms_gather"),
                     4 * (tot("trav_large") - tot("trav_hub") + tot("incid_large"))
                     + 12 * tot("incid_large") + 4 * tot("hub_words"),
                     tot("trav_large")),
        "k_color_wave": (tot("ms_color"),
                         4 * (tot("trav_total") - tot("trav_large") + tot("incid_total")
                              - tot("incid_large")) + 12 * (tot("incid_total") - tot("incid_large"))
                         + 28 * (tot("w_total") - tot("w_large")),
                         tot("trav_total") - tot("trav_large")),
    }
    if batched:
        # the persistent kernel: 8 B per traversed two-hop entry (the member id
        # and its color), 12 B per incidence (a_idx and the b_ptr pair), 28 B
        # per work-queue entry (queue, a_ptr pair, sums, stage, colors) and,
        # per round, 8 B per CSC entry for the per-net conflict detection
        det = sum(g.nnz * r for g, r in zip(graphs, last_rounds))
        kern = {"k_batch": (tot("ms_color"), 8 * tot("trav_total") + 12 * tot("incid_total")
                            + 28 * tot("w_total") + 8 * det * args.steps,
                            tot("trav_total"))}
        n_launch = args.steps
    dom = max(kern, key=lambda k: kern[k][0])
    dom_ms, dom_bytes, dom_entries = kern[dom]
    peak, peak_kind = peaks()
    achieved = dom_bytes / (dom_ms / 1000.0) / 1e9 if dom_ms > 0 else 0.0
    # the vertex-based formulation's model: 8 B (an index and a gathered
    # color) per traversed two-hop entry, hub entries included although they
    # are read as bitmaps
    eff8 = 8 * dom_entries / (dom_ms / 1000.0) / 1e9 if dom_ms > 0 else 0.0
    phase_ms = {k: tot(k) / args.steps
                for k in ("ms_setup", "ms_gather", "ms_color", "ms_publish", "ms_detect")}
    bpl = dom_bytes / max(n_launch, 1)
    traffic = kernel_traffic("k_gather_w" if dom == "k_gather" else dom, bpl)

    # end to end through the public API: H2D of the graph from pinned host
    # memory, coloring, D2H of the colors, every step
    host = []
    graphs_e2e = [] if (args.no_e2e or d2) else graphs
    for g in graphs_e2e:
        arrs = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
                for a in (g.a_ptr, g.a_idx, g.b_ptr, g.b_idx)]
        host.append(arrs)
    out_host = [torch.empty(g.n_a, dtype=torch.int32).pin_memory() for g in graphs_e2e]
    h2d = sum(a.numel() * 4 for arrs in host for a in arrs)
    d2h = sum(g.n_a * 4 for g in graphs_e2e)

    def e2e_step():
        for (hg, dg) in zip(host, dgs):
            for src, dst in zip(hg, (dg.a_ptr, dg.a_idx, dg.b_ptr, dg.b_idx)):
                dst.copy_(src, non_blocking=True)
        if batched:
            bg.bgpc_color_batched(ctx, dgs, colors)
        else:
            for dg, c in zip(dgs, colors):
                bg.bgpc_color(ctx, dg, c)
        for oh, c in zip(out_host, colors):
            oh.copy_(c, non_blocking=True)

    e2e = None
    if graphs_e2e:
        for _ in range(max(1, args.warmup)):
            e2e_step()
        barrier(world)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        e_ms = max_over_ranks(world, e0.elapsed_time(e1), dev)
        e2e = {"value": world * entries_step * args.steps / (e_ms / 1000.0), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
        for oh, c in zip(out_host, colors):
            assert torch.equal(oh, c.cpu())

    jac = args.workload == "jacobian"
    records = seq_records() if rank == 0 else []
    d2gc = None
    if rank == 0 and jac and not args.no_d2gc:
        d2gc = d2gc_report(bg, ctx, dev, steps=3, warmup=1, records=records)

    schedules = None
    if rank == 0 and jac:
        schedules = schedule_report(bg, ctx, dgs, graphs, 3, records)

    learned = None
    if rank == 0 and not args.no_learned and jac:
        learned = learned_order_report(bg, ctx, dev, dgs[1])

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and jac:
        import oracle
        oracle.build()
        cpu = oracle_sample(graphs, args.cpu_budget, os.cpu_count() or 1)
        cpu = {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample", "per_graph",
                                   "cpu_model")}

    if rank == 0:
        per_graph = []
        if batched:
            st = all_stats[-1][0]
            per_graph.append({"graphs": len(graphs), "n_a": sum(g.n_a for g in graphs),
                              "nnz": sum(g.nnz for g in graphs),
                              "E2": sum(e2_of(g) for g in graphs),
                              "rounds_max": st["rounds"], "colors_max": st["colors"],
                              "w_per_round": st["w_per_round"][:12],
                              "trav_total": st["trav_total"], "trav_large": st["trav_large"],
                              "pieces": st["pieces_total"]})
        for g, st, dg, c in ([] if batched else zip(graphs, all_stats[-1], dgs, colors)):
            rec = {"graph": g.name, "n_a": n_of(g), "nnz": g.nnz, "E2": e2_of(g),
                   "rounds": st["rounds"], "colors": st["colors"],
                   "w_per_round": st["w_per_round"][:12],
                   "trav_total": st["trav_total"], "inflation": st["trav_total"] / e2_of(g),
                   "trav_large": st["trav_large"], "pieces": st["pieces_total"],
                   "trav_hub": st["trav_hub"], "hub_pairs": st["hub_pairs"],
                   "hub_words": st["hub_words"]}
            if not d2:
                sizes = np.diff(g.b_ptr)
                rec["colors_lower_bound"] = int(sizes.max()) if sizes.size else 0
                seq = seq_for(records, graph_sha1(g), "FF")
                rec["colors_seq"] = seq["colors"] if seq else None
                rec["colors_vs_seq"] = st["colors"] / seq["colors"] if seq else None
                _, bal = bg.bgpc_color_sets(ctx, c, st["colors"])
                rec["balance"] = bal
                rec["seq_balance"] = seq
            per_graph.append(rec)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload],
                       "l2": "inputs larger than L2 (no flush)",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "graphs": per_graph, "phase_ms_per_step": phase_ms},
            # the same step measured two more ways: useful two-hop edges (one
            # full sweep E2 per graph) per second, and traversed entries
            # without the hub-net entries that are read as color bitmaps
            "E2_per_s": world * e2_step * args.steps / (ms_max / 1000.0),
            "nonhub_entries_per_s": world * (entries_step - hub_step) * args.steps
            / (ms_max / 1000.0),
            "roofline": {"bound": "hbm", "kernel": dom,
                         "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind,
                         "traffic": traffic,
                         "bytes_per_launch": bpl,
                         "ms_per_launch": dom_ms / max(n_launch, 1),
                         "launches": n_launch,
                         "frac_8B_per_entry": eff8 / peak,
                         "other": {k: {"ms_per_step": v[0] / args.steps,
                                       "GB_s": (v[1] / (v[0] / 1000.0) / 1e9) if v[0] else 0.0}
                                   for k, v in kern.items()}},
            "e2e": e2e,
            "gpu_launches": launches,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "schedules": schedules,
            "d2gc_rmat22": d2gc,
            "learned_order": learned,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-d2gc", action="store_true")
    ap.add_argument("--workload", default="jacobian", choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
