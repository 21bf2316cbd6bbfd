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
    # the batched configuration: 512 independent graphs, one bgpc_color_batched call
    "batch512": ("512 graphs, |V_A| log-uniform [1e3,1e6], |V_B| = |V_A|*U[0.5,2], degree "
                 "Poisson(8) clipped to [1,64]; RS(64,16,64) first fit, id order, one batched call"),
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
    return [gg.stencil9(1024), gg.chung_lu(1 << 22, 16.0, 50000.0, 2.1, seed=2)]


def e2_of(g) -> int:
    s = np.diff(g.b_ptr).astype(np.int64)
    return int((s * (s - 1)).sum())


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
    nothing colored yet), as many as fit the time budget."""
    import oracle as O
    stencil, cl = graphs
    t0 = time.perf_counter()
    r = O.rs_color(stencil, O.FF, nthreads=nthreads)
    t_st = time.perf_counter() - t0
    entries = int(r.trav_per_round.sum())
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
    while spent < budget_s and chunks_done < nch:
        ch = order[chunks_done:chunks_done + batch].astype(np.int32)
        t1 = time.perf_counter()
        O.rs_chunks(cl, S, W, ch, O.FF, chunk=64, big_net=64, nthreads=nthreads)
        spent += time.perf_counter() - t1
        for j in ch:
            entries += int(per_vertex[j * 64:(j + 1) * 64].sum())
        chunks_done += len(ch)
    return {"value": entries / spent, "unit": UNIT, "cores": nthreads, "kind": "oracle",
            "sample": (f"full RS replay of stencil9 1024x1024 ({int(r.trav_per_round.sum())} "
                       f"entries, {r.rounds} rounds) + {chunks_done} of {nch} round-1 chunks of "
                       f"the Chung-Lu graph ({nthreads} threads, {spent:.1f} s)"),
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
                             "sample": s["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- GPU leg

def learned_order_report(bg, ctx, dev, chung_lu_dg):
    """The learned vertex order (features -> MLP -> rank) against id order:
    trained on 16 graphs of the batched workload (seed 23), evaluated on the
    Chung-Lu 2^22 graph and on 64 fresh graphs of the batched workload
    (seed 29, |V_A| log-uniform in [1e3, 1e6]).  Reports colors used."""
    import torch
    import graphgen as gg
    train = [bg.DeviceGraph.from_host(gg.batch_graph(23, i, lo=1e3, hi=1e5), dev)
             for i in range(16)]
    t0 = time.time()
    mlp, losses = bg.train_order(ctx, train, torch.from_numpy(gg.mlp_init(7)).to(dev),
                                 steps=300, lr=3e-3)
    torch.cuda.synchronize()
    t_train = time.time() - t0

    def colors(dg, rank=None):
        _, st, _ = bg.bgpc_color(ctx, dg, rank=rank)
        return st["colors"]

    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record()
    rank = bg.learned_rank(ctx, chung_lu_dg, mlp)
    s1.record()
    torch.cuda.synchronize()
    cl = {"colors_id": colors(chung_lu_dg), "colors_learned": colors(chung_lu_dg, rank),
          "ms_order": s0.elapsed_time(s1)}
    fresh_id, fresh_l = [], []
    for i in range(64):
        dg = bg.DeviceGraph.from_host(gg.batch_graph(29, i), dev)
        fresh_id.append(colors(dg))
        fresh_l.append(colors(dg, bg.learned_rank(ctx, dg, mlp)))
    return {"model": "MLP 8-64-64-1, bf16 weights, fp32 arithmetic, Adam",
            "train": {"graphs": 16, "steps": len(losses), "loss_first": losses[0],
                      "loss_last": losses[-1], "seconds": t_train},
            "chung_lu_2^22": cl,
            "fresh_batch_graphs": {"graphs": 64, "colors_id_mean": float(np.mean(fresh_id)),
                                   "colors_learned_mean": float(np.mean(fresh_l)),
                                   "fewer_colors": int(sum(a > b for a, b in zip(fresh_id, fresh_l))),
                                   "more_colors": int(sum(a < b for a, b in zip(fresh_id, fresh_l)))}}


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
    ctx = bg.Context(local)
    dgs = [bg.DeviceGraph.from_host(g, dev) for g in graphs]
    colors = [torch.empty(g.n_a, dtype=torch.int32, device=dev) for g in graphs]
    stream = torch.cuda.current_stream()

    batched = args.workload == "batch512"

    def step(profile=False):
        if batched:
            _, st, _, _ = bg.bgpc_color_batched(ctx, dgs, colors, profile=profile)
            return [st]
        sts = []
        for dg, c in zip(dgs, colors):
            _, st, _ = bg.bgpc_color(ctx, dg, c, profile=profile)
            sts.append(st)
        return sts

    for _ in range(args.warmup):
        step()
    # correctness of the timed configuration: valid colorings
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
                     + 12 * tot("incid_large") + 4 * tot("hub_words")),
        "k_color_wave": (tot("ms_color"),
                         4 * (tot("trav_total") - tot("trav_large") + tot("incid_total")
                              - tot("incid_large")) + 12 * (tot("incid_total") - tot("incid_large"))
                         + 28 * (tot("w_total") - tot("w_large"))),
    }
    dom = max(kern, key=lambda k: kern[k][0])
    dom_ms, dom_bytes = kern[dom]
    peak, peak_kind = peaks()
    achieved = dom_bytes / (dom_ms / 1000.0) / 1e9 if dom_ms > 0 else 0.0
    phase_ms = {k: tot(k) / args.steps
                for k in ("ms_setup", "ms_gather", "ms_color", "ms_publish", "ms_detect")}

    # end to end through the public API: H2D of the graph from pinned host
    # memory, coloring, D2H of the colors, every step
    host = []
    if args.no_e2e:
        graphs_e2e = []
    else:
        graphs_e2e = graphs
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

    learned = None
    if rank == 0 and not args.no_learned and args.workload == "jacobian":
        learned = learned_order_report(bg, ctx, dev, dgs[1])

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "jacobian":
        import oracle
        oracle.build()
        cpu = oracle_sample(graphs, args.cpu_budget, os.cpu_count() or 1)
        cpu = {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")}

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
        for g, st in ([] if batched else zip(graphs, all_stats[-1])):
            per_graph.append({"graph": g.name, "n_a": g.n_a, "nnz": g.nnz, "E2": e2_of(g),
                              "rounds": st["rounds"], "colors": st["colors"],
                              "w_per_round": st["w_per_round"][:12],
                              "trav_total": st["trav_total"],
                              "trav_large": st["trav_large"], "pieces": st["pieces_total"],
                              "trav_hub": st["trav_hub"], "hub_pairs": st["hub_pairs"],
                              "hub_words": st["hub_words"]})
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload],
                       "l2": "inputs larger than L2 (no flush)",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "graphs": per_graph, "phase_ms_per_step": phase_ms},
            "roofline": {"bound": "hbm", "kernel": dom,
                         "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind,
                         "traffic": None,
                         "bytes_per_launch": dom_bytes / max(n_launch, 1),
                         "ms_per_launch": dom_ms / max(n_launch, 1),
                         "launches": n_launch,
                         "other": {k: {"ms_per_step": v[0] / args.steps,
                                       "GB_s": (v[1] / (v[0] / 1000.0) / 1e9) if v[0] else 0.0}
                                   for k, v in kern.items()}},
            "e2e": e2e,
            "gpu_launches": launches,
            "cpu_baseline": cpu,
            "clocks": clocks,
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
    ap.add_argument("--workload", default="jacobian", choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
