#!/usr/bin/env python3
"""Benchmark of the Tensor Data Platform hot path on one B300 (or N replicas).

Headline step: the shipping-priority query plan on a 60M-row fact table and a
15M-row dimension table (dimension filter -> hash build; fact filter fused
into the probe with a gather; sort-based GROUP BY key of
SUM(price*(100-disc)); top-10), all on synthetic seeded data.  value = fact
rows per second over the whole job.

The same run also times, on their own inputs: the pricing-summary plan
(filter + small-domain group-by over 60M rows), the three-table join chain
(100M probe rows, fused probe + group-by), the soft query forward+backward
(10M rows) and, when built, the glyph-CNN trainable-query training step.

Flags: --gpus N --steps K --warmup W [--impl reference] [--plans all|main]
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

import gen  # noqa: E402

N_FACT = 60_000_000
N_DIM = 15_000_000
SEED2 = gen.BASE_SEED + 1
WORKLOAD = "shipping-priority plan: 60M-row fact x 15M-row dimension, filter+join+group-by+top-10"


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6400.0), "measured"
    return 6400.0, "fallback"


def shipping_inputs():
    fact = gen.fact_table(N_FACT, N_DIM, SEED2, cols=("key", "price", "disc", "date"))
    dim = gen.dim_table(N_DIM, SEED2, cols=("key", "segment"))
    return fact, dim


# --------------------------------------------------------------- reference

def cpu_shipping_sample(scale: int):
    """The oracle (plain C, single thread) on a 1/scale sample of the
    shipping-priority workload (same generator, key range scaled with it).
    Returns (fact rows, seconds)."""
    from oracle import relational as R
    nf, nd = N_FACT // scale, N_DIM // scale
    fact = gen.fact_table(nf, nd, SEED2 + 1000 + scale, cols=("key", "price", "disc", "date"))
    dim = gen.dim_table(nd, SEED2 + 1000 + scale, cols=("key", "segment"))
    t0 = time.perf_counter()
    bsel = R.filter([(dim["segment"], "==", 2)], nd)
    psel = R.filter([(fact["date"], ">", 1200)], nf)
    prow, brow, _ = R.join(dim["key"], fact["key"], bsel=bsel, psel=psel)
    keys, aggs = R.groupby([fact["key"]], [("sum_mul_kminus", fact["price"], fact["disc"], 100)], nf, sel=prow)
    R.topk(aggs[:, 0], keys[:, 0], 10)
    return nf, time.perf_counter() - t0


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    scale = 20
    rows, secs = [], []
    for _ in range(args.warmup):
        cpu_shipping_sample(scale)
    for _ in range(args.steps):
        r, s = cpu_shipping_sample(scale)
        rows.append(r)
        secs.append(s)
    v = sum(rows) / sum(secs)
    line = {
        "impl": "reference", "metric": "fact rows/s (shipping-priority plan)", "value": v, "unit": "rows/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * sum(secs) / len(secs), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "fact_rows": N_FACT, "dim_rows": N_DIM, "parallelism": "replicas"},
        "cpu_baseline": {"value": v, "unit": "rows/s", "cores": 1, "kind": "oracle",
                         "sample": "1/%d of the workload per step (%d fact rows, %d dimension rows), plain C "
                                   "oracle, one thread" % (scale, N_FACT // scale, N_DIM // scale)},
        "e2e": {"value": v, "unit": "rows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- traffic

# DRAM bytes (read + write) of a stage's kernel from an ncu capture kept in
# profiles/, per fact row of the capture's workload, and the source file it was
# built from.  The capture ran the plan at 1/4 scale; every term of the
# probe's traffic grows with the fact rows, so it is scaled by them.
TRAFFIC = {
    "join_probe": {"bytes_per_fact_row": (328.591104e6 + 7.65696e6) / 15e6,
                   "src": "paper_2211_02753_b300/csrc/join.cu", "sha1": "3fbda6a2fcd7",
                   "capture": "profiles/join_probe_kernel_15M_fact_rows.md"},
}


def measured_traffic(stage: str):
    """Per-launch DRAM bytes of the stage at full size, or None when there is
    no capture or the kernel source changed since it was taken."""
    import hashlib
    t = TRAFFIC.get(stage)
    if t is None:
        return None
    with open(os.path.join(ROOT, t["src"]), "rb") as f:
        if hashlib.sha1(f.read()).hexdigest()[:12] != t["sha1"]:
            return None
    return t["bytes_per_fact_row"] * N_FACT


# ------------------------------------------------------------- multi-rank

def job_rate(units_per_rank: float, ms_local: float, world: int, device):
    """Whole-job rate of `world` replicas: every rank processes
    units_per_rank per step; the step time is the MAX over ranks (the slowest
    replica bounds the job).  Returns (ms_per_step, units per second)."""
    import torch
    import torch.distributed as dist
    ms = float(ms_local)
    if world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, units_per_rank * world / (ms / 1000.0)


# ------------------------------------------------------------------ clocks

class ClockSampler:
    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + q, "--format=csv,noheader,nounits",
                                          "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
            return
        # wait for the first sample so that the timed region is covered
        t_end = time.time() + 10
        while time.time() < t_end and os.path.getsize(self.path) == 0:
            time.sleep(0.05)

    def stop(self, gpu_index: int):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9 or not p[0].isdigit() or int(p[0]) != gpu_index:
                    continue
                try:
                    sm.append(float(p[1]))
                    smax.append(float(p[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, p[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------- GPU arm

def run_gpu(args):
    import torch
    import torch.distributed as dist
    from paper_2211_02753_b300 import ops, plans
    from paper_2211_02753_b300 import _lib

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _lib.lib()  # fail loudly if the library is missing

    def barrier():
        if world > 1:
            dist.barrier()

    hbm_peak, peak_kind = load_peaks()

    # ---- headline: shipping-priority plan
    fact_h, dim_h = shipping_inputs()
    fact = {k: torch.from_numpy(v).to(dev) for k, v in fact_h.items()}
    dim = {k: torch.from_numpy(v).to(dev) for k, v in dim_h.items()}
    plan = plans.ShippingPriority(fact, dim)
    stream = torch.cuda.current_stream()
    for _ in range(max(3, args.warmup)):
        out = plan.run()
    torch.cuda.synchronize()
    ops.check(plan.status, "shipping-priority plan")
    nmatch = int(out["nmatch"].item())
    ngroups = int(out["ngroups"].item())

    # stage timing (CUDA events on the launching stream) for the roofline
    def stage_times(reps=3):
        ev = []
        for _ in range(reps):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
            e[0].record(stream)
            ops.join_build([dim["key"], dim["segment"]], 0, preds=[(1, "==", 2)], nslots=plan.nslots,
                           table=plan.table, status=plan.status)
            e[1].record(stream)
            pr = ops.join_probe(plan.table, [fact["key"], fact["date"], fact["price"], fact["disc"]], 0,
                                preds=[(1, ">", 1200)], gather=[0, 2, 3], capacity=plan.cap, rowids=False,
                                payload=False, status=plan.status)
            e[2].record(stream)
            kc, pc, dc = pr["gathered"]
            gb = ops.groupby_agg([ops.Col(kc, 1, N_DIM), pc, dc], [0], [("sum_mul_kminus", 1, 2, 100)],
                                 n=plan.cap, nsel=pr["count"], strategy=plan.groupby_strategy, capacity=plan.cap,
                                 status=plan.status)
            e[3].record(stream)
            ops.topk(gb["aggs"][0], gb["keys"][0], 10, d_n=gb["ngroups"], status=plan.status)
            e[4].record(stream)
            torch.cuda.synchronize()
            ev.append([e[i].elapsed_time(e[i + 1]) for i in range(4)])
        return [statistics.median(x[i] for x in ev) for i in range(4)]

    st_ms = stage_times()

    # the timed step: the plan captured once as a CUDA graph and replayed
    # (the same kernels; no host work between launches)
    step = plans.Graphed(plan)
    out = step.run()
    torch.cuda.synchronize()
    ops.check(plan.status, "shipping-priority plan (graph)")
    assert int(out["nmatch"].item()) == nmatch and int(out["ngroups"].item()) == ngroups

    # timed region
    sampler = ClockSampler()
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        out = step.run()
    t1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop(local)
    ms, value = job_rate(N_FACT, t0.elapsed_time(t1) / args.steps, world, dev)
    ops.check(plan.status, "shipping-priority plan")

    # ---- e2e: host (pinned) buffers in, top-10 out, every step
    pin_f = {k: torch.from_numpy(v).pin_memory() for k, v in fact_h.items()}
    pin_d = {k: torch.from_numpy(v).pin_memory() for k, v in dim_h.items()}
    h2d = sum(v.numel() * v.element_size() for v in list(pin_f.values()) + list(pin_d.values()))
    out_v = torch.empty(10, dtype=torch.int64).pin_memory()
    out_k = torch.empty(10, dtype=torch.int32).pin_memory()
    d2h = 10 * 8 + 10 * 4

    def e2e_step():
        for k in fact:
            fact[k].copy_(pin_f[k], non_blocking=True)
        for k in dim:
            dim[k].copy_(pin_d[k], non_blocking=True)
        o = step.run()
        out_v.copy_(o["top_vals"], non_blocking=True)
        out_k.copy_(o["top_keys"], non_blocking=True)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e2e_steps = max(1, min(args.steps, 5))
    e0.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    e2e_value = N_FACT * world / (e2e_ms / 1000.0)

    # ---- kernel launches per step (profiler on one extra, untimed step)
    launches_per_step = None
    try:
        from torch.profiler import ProfilerActivity, profile
        with profile(activities=[ProfilerActivity.CUDA]) as prof:
            plan.run()
            torch.cuda.synchronize()
        names = [e.name for e in prof.events() if e.device_type.name == "CUDA"]
        launches_per_step = sum(1 for n in names if "tdp::" in n)
    except Exception:
        launches_per_step = None

    # ---- roofline of the dominant stage
    stage_names = ["join_build", "join_probe", "groupby", "topk"]
    sel_f = float(np.mean(fact_h["date"] > 1200))
    probe_rows = N_FACT * sel_f
    algo = {
        # build: dim segment (1 B) for every row + key (4 B) for matches + table slot writes (8 B/slot fill +
        # 8 B per insert)
        "join_build": N_DIM * 1 + N_DIM * 0.2 * 4 + plan.nslots * 8 + N_DIM * 0.2 * 8,
        # probe: date (4 B) every row; key (4 B) of qualifying rows; one 8-byte slot per lookup; price/disc
        # (16 B) of matches; key/price/disc written for matches (20 B)
        "join_probe": N_FACT * 4 + probe_rows * 4 + probe_rows * 8 + nmatch * 16 + nmatch * 20,
        # partitioned group-by: count (key 4 B), scatter (key, price, disc 20 B in; gid + value 12 B out),
        # bucket reduce (12 B in), groups out (key 4 B + sum 8 B)
        "groupby": nmatch * (4 + 20 + 12 + 12) + ngroups * 12,
        "topk": ngroups * 12,
    }
    dom = int(np.argmax(st_ms))
    dom_name = stage_names[dom]
    achieved = algo[dom_name] / (st_ms[dom] / 1000.0) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": measured_traffic(dom_name), "kernel": dom_name,
                "peak_kind": peak_kind + " (copy bandwidth)",
                "stages_ms": dict(zip(stage_names, st_ms)),
                "stages_algo_gbs": {k: algo[k] / (t / 1000.0) / 1e9 for k, t in zip(stage_names, st_ms)}}

    line = {
        "metric": "fact rows/s (shipping-priority plan)", "value": value, "unit": "rows/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "fact_rows": N_FACT, "dim_rows": N_DIM, "matches": nmatch,
                   "groups": ngroups, "parallelism": "replicas" if world > 1 else "single-gpu",
                   "l2": "inputs larger than L2 (1.5 GB of columns per step)",
                   "launch": "each step one replay of the plan captured as a CUDA graph"},
        "roofline": roofline,
        "e2e": {"value": e2e_value, "unit": "rows/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e2e_ms},
        "gpu_launches": (launches_per_step * args.steps) if launches_per_step is not None else None,
        "gpu_launches_per_step": launches_per_step,
        "clocks": clocks,
    }
    del fact, dim, plan, pin_f, pin_d
    torch.cuda.empty_cache()

    if args.plans == "all":
        line["plans"] = other_plans(dev, stream, hbm_peak, args)

    if rank == 0:
        # CPU baseline: the oracle on a bounded sample (rank 0, N=1 semantics)
        scale = 20
        r, s = cpu_shipping_sample(scale)
        line["cpu_baseline"] = {"value": r / s, "unit": "rows/s", "cores": 1, "kind": "oracle",
                                "sample": "1/%d of the workload (%d fact rows, %d dimension rows), plain C "
                                          "oracle, one thread, %.1f s" % (scale, r, N_DIM // scale, s)}
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def _time(fn, stream, steps):
    import torch
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


def _time_graph(fn, stream, steps):
    """_time of replays of fn captured once as a CUDA graph: the same library
    kernels without host work between the launches.  fn neither synchronises
    nor allocates outside torch's caching allocator (every op of the
    relational and soft plans); its outputs are rewritten by each replay."""
    import torch
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):  # workspaces and output pools settle before capture
        for _ in range(3):
            fn()
    stream.wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fn()
    return _time(g.replay, stream, steps)


def other_plans(dev, stream, hbm_peak, args):
    import torch
    from paper_2211_02753_b300 import ops, plans
    res = {}
    steps = max(3, args.steps)
    # pricing summary at 60M rows
    t = gen.fact_table(N_FACT, N_DIM, SEED2, cols=("flag", "status", "qty", "price", "disc", "date"))
    sel = float(np.mean(t["date"] <= 2460))
    td = {k: torch.from_numpy(v).to(dev) for k, v in t.items()}
    td["key"] = None
    del t
    # standalone filter with stream compaction (row ids) over the 60M-row date column
    fout = {}

    def run_filter():
        fout["o"] = ops.filter([td["date"]], [(0, "<=", 2460)], rowids=True)

    ms = _time_graph(run_filter, stream, steps)
    nsel = int(fout["o"]["count"].item())
    fbytes = N_FACT * 4 + nsel * 4
    res["filter_60M"] = {"ms": ms, "rows_per_s": N_FACT / (ms / 1e3), "selected": nsel,
                         "algo_gbs": fbytes / (ms / 1e3) / 1e9, "frac_hbm": fbytes / (ms / 1e3) / 1e9 / hbm_peak}
    for strategy in ("small_domain", "sort"):
        p = plans.PricingSummary(td, strategy)
        ms = _time_graph(lambda: p.run(), stream, steps if strategy == "small_domain" else 3)
        bpr = plans.PricingSummary.bytes_per_row(sel)
        res["pricing_summary_60M_" + strategy] = {"ms": ms, "rows_per_s": N_FACT / (ms / 1e3),
                                                  "algo_gbs": N_FACT * bpr / (ms / 1e3) / 1e9,
                                                  "frac_hbm": N_FACT * bpr / (ms / 1e3) / 1e9 / hbm_peak}
    del td
    torch.cuda.empty_cache()
    # join chain (100M probe rows)
    d = gen.chain_tables(100_000_000, 10_000_000, 1_000_000, gen.BASE_SEED + 2)
    dd = {k: torch.from_numpy(v.astype(np.int32) if k == "probe_fk" else v).to(dev) for k, v in d.items()}
    del d
    jc = plans.JoinChain(dd)
    ms = _time_graph(lambda: jc.run(), stream, steps)
    out = jc.run()
    torch.cuda.synchronize()
    ops.check(jc.status, "join chain")
    algo = 100e6 * (4 + 8 + 8) + 10e6 * (4 + 4 + 8 + 8) + 1e6 * 8
    res["join_chain_100M"] = {"ms": ms, "rows_per_s": 100e6 / (ms / 1e3), "algo_gbs": algo / (ms / 1e3) / 1e9,
                              "frac_hbm": algo / (ms / 1e3) / 1e9 / hbm_peak,
                              "groups": int(out["ngroups"].item())}
    del dd, jc
    torch.cuda.empty_cache()
    # soft query fwd+bwd (10M rows)
    s = gen.soft_table(10_000_000, 1024, gen.BASE_SEED + 3)
    sd = {k: torch.from_numpy(v).to(dev) for k, v in s.items()}
    sq = plans.SoftQuery(sd)
    ms = _time_graph(lambda: sq.run(), stream, steps)
    algo = 10e6 * 24
    res["soft_query_10M_fwd_bwd"] = {"ms": ms, "rows_per_s": 10e6 / (ms / 1e3), "algo_gbs": algo / (ms / 1e3) / 1e9,
                                     "frac_hbm": algo / (ms / 1e3) / 1e9 / hbm_peak}
    # the individual soft kernels: aggregation forward / backward (12 B/row
    # each), soft filter forward (12 B/row: x, gid in, mask out) and backward
    # (16 B/row: x, gid, grad_mask in, grad_x out)
    th, tau = sq.theta, sq.tau
    gm = torch.ones_like(sd["x"])
    for name, fn, bpr in (
            ("soft_agg_fwd_10M", lambda: ops.soft_agg_fwd(sd["x"], sd["v"], sd["gid"], th, tau), 12),
            ("soft_agg_bwd_10M", lambda: ops.soft_agg_bwd(sd["x"], sd["v"], sd["gid"], th, tau, sq.gS, sq.gC), 12),
            ("soft_filter_fwd_10M", lambda: ops.soft_filter_fwd(sd["x"], sd["gid"], th, tau), 12),
            ("soft_filter_bwd_10M", lambda: ops.soft_filter_bwd(sd["x"], sd["gid"], th, tau, gm), 16)):
        ms = _time_graph(fn, stream, steps)
        res[name] = {"ms": ms, "rows_per_s": 10e6 / (ms / 1e3), "algo_gbs": 10e6 * bpr / (ms / 1e3) / 1e9,
                     "frac_hbm": 10e6 * bpr / (ms / 1e3) / 1e9 / hbm_peak}
    del sd, sq
    torch.cuda.empty_cache()
    res["trainable_query_glyph_cnn"] = glyph_plan(dev, stream, args)
    return res


def glyph_plan(dev, stream, args):
    """Trainable glyph query: train steps/s (batch 256 grids = 4096 cells),
    exact-query steps/s on the same GPU, and the query-level accuracy reached
    after a fixed training budget."""
    import torch
    from oracle import cnn as O  # targets: the exact query on the true labels
    from oracle import soft
    from paper_2211_02753_b300 import cnn
    tr_img, tr_lab = gen.glyph_grids(4096, gen.BASE_SEED + 4)
    te_img, te_lab = gen.glyph_grids(1024, gen.BASE_SEED + 104)
    targets = torch.from_numpy(O.targets_from_labels(tr_lab).astype(np.float32)).to(dev)
    g_tr = torch.from_numpy(tr_img).to(dev)
    g_te = torch.from_numpy(te_img).to(dev)
    q = cnn.GlyphQuery(gen.cnn_params(gen.BASE_SEED + 5), dev, lr=1e-3, warmup=400)
    B = 256
    nb = 4096 // B

    def step(i):
        j = (i % nb) * B
        return q.train_step(g_tr[j:j + B], targets[j:j + B])

    for i in range(3):
        step(i)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    n_timed = max(20, args.steps)
    a.record(stream)
    for i in range(n_timed):
        step(3 + i)
    b.record(stream)
    torch.cuda.synchronize()
    train_ms = a.elapsed_time(b) / n_timed
    # finish a fixed training budget, then evaluate the exact query
    budget = 1600
    for i in range(3 + n_timed, budget):
        step(i)
    torch.cuda.synchronize()
    gq = g_te[:B]
    for _ in range(3):
        q.exact_query(gq)
    a.record(stream)
    for _ in range(n_timed):
        q.exact_query(gq)
    b.record(stream)
    torch.cuda.synchronize()
    infer_ms = a.elapsed_time(b) / n_timed
    labels, cnt, rsum = q.exact_query(g_te)
    ec, er = soft.exact_groupby(te_lab)
    ok = np.all(cnt.cpu().numpy() == ec, axis=1) & np.all(rsum.cpu().numpy() == er, axis=1)
    cell_acc = float((labels.cpu().numpy().reshape(-1, 4, 4) == te_lab).mean())
    flops_fwd = 4096 * 2 * (26 * 26 * 32 * 9 + 24 * 24 * 64 * 288 + 9216 * 128 + 128 * 10)
    return {"train_ms": train_ms, "train_steps_per_s": 1000.0 / train_ms, "exact_query_ms": infer_ms,
            "exact_query_steps_per_s": 1000.0 / infer_ms, "batch_grids": B, "training_steps": budget,
            "query_accuracy": float(ok.mean()), "cell_accuracy": cell_acc,
            "train_tflops": 3 * flops_fwd / (train_ms / 1e3) / 1e12}


def run_only(args):
    """One plan at 1/scale of its size, `steps` times after `warmup` runs, and
    a one-line timing (CUDA events).  Used for profiler captures of a small
    case; not the benchmark line."""
    import torch
    from paper_2211_02753_b300 import cnn, ops, plans
    from oracle import cnn as O  # glyph targets: the exact query on true labels
    dev = torch.device("cuda", 0)
    sc = max(1, args.scale)
    if args.only in ("shipping", "shipping_sep"):
        f, d = (gen.fact_table(N_FACT // sc, N_DIM // sc, SEED2, cols=("key", "price", "disc", "date")),
                gen.dim_table(N_DIM // sc, SEED2, cols=("key", "segment")))
        p = plans.ShippingPriority({k: torch.from_numpy(v).to(dev) for k, v in f.items()},
                                   {k: torch.from_numpy(v).to(dev) for k, v in d.items()},
                                   groupjoin=args.only == "shipping")
        fn = p.run
    elif args.only in ("pricing", "pricing_sort", "filter"):
        t = gen.fact_table(N_FACT // sc, N_DIM // sc, SEED2, cols=("flag", "status", "qty", "price", "disc", "date"))
        td = {k: torch.from_numpy(v).to(dev) for k, v in t.items()}
        if args.only == "filter":
            fn = lambda: ops.filter([td["date"]], [(0, "<=", 2460)])  # noqa: E731
        else:
            fn = plans.PricingSummary(td, "sort" if args.only == "pricing_sort" else "small_domain").run
    elif args.only == "chain":
        dd = gen.chain_tables(100_000_000 // sc, 10_000_000 // sc, 1_000_000 // sc, gen.BASE_SEED + 2)
        fn = plans.JoinChain({k: torch.from_numpy(v.astype(np.int32) if k == "probe_fk" else v).to(dev)
                              for k, v in dd.items()}).run
    elif args.only == "soft":
        s = gen.soft_table(10_000_000 // sc, 1024, gen.BASE_SEED + 3)
        fn = plans.SoftQuery({k: torch.from_numpy(v).to(dev) for k, v in s.items()}).run
    else:  # glyph: one training step of the trainable query
        g = max(16, 256 // sc)
        img, lab = gen.glyph_grids(g, gen.BASE_SEED + 4)
        q = cnn.GlyphQuery(gen.cnn_params(gen.BASE_SEED + 5), dev)
        gi = torch.from_numpy(img).to(dev)
        tg = torch.from_numpy(O.targets_from_labels(lab).astype(np.float32)).to(dev)
        fn = lambda: q.train_step(gi, tg)  # noqa: E731
    for _ in range(args.warmup):
        fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        fn()
    b.record()
    torch.cuda.synchronize()
    print(json.dumps({"only": args.only, "scale": sc, "ms": a.elapsed_time(b) / max(1, args.steps)}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--plans", default="all", choices=["all", "main"])
    ap.add_argument("--only", default=None,
                    choices=["shipping", "shipping_sep", "pricing", "pricing_sort", "filter", "chain", "soft",
                             "glyph"],
                    help="profiling mode: run one plan at 1/--scale size and print its time only")
    ap.add_argument("--scale", type=int, default=1)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.only:
        return run_only(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
