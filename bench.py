#!/usr/bin/env python3
"""Benchmark of the Tensor Data Platform hot path on one B300 (or N replicas).

Headline step: the shipping-priority query plan on a 60M-row fact table and a
15M-row dimension table -- dimension WHERE segment = 2, fact WHERE date >
1200, inner join on key, GROUP BY key SUM(price*(100-disc)), top-10 -- run as
one group-join (build: rank code of the dimension keys; probe: fact rows
accumulate into their group; finish: groups in key order and the top-10), on
synthetic seeded data.  value = fact rows per second over the whole job.

The same run also measures, on their own inputs and each with a `roofline`
object and a `cpu_baseline` (the oracle on the host cores, single-threaded
and OpenMP row-partitioned where it has that form): the standalone filter;
the pricing summary (small-domain and onesweep sort group-by); the shipping
plan on the separate build -> probe -> group-by path (partition and sort
group-by); the three-table join chain (fused probe + group-by, and probe ->
sort group-by); the N:M join; dictionary codes of a string column and a
GROUP BY over two coded columns; the soft query forward/backward kernels;
the glyph-CNN and Digit x Size trainable queries with their exact queries;
learning from label proportions (the 64M-row step and the census error by
bag size); the soft top-k.

Flags: --gpus N --steps K --warmup W [--impl reference] [--plans all|main]
[--only PLAN --scale S: one plan at 1/S of its size, for profiler captures]
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
        return d.get("hbm_gbs", 6400.0), d.get("bf16_tflops_sustained", 1400.0), "measured"
    return 6400.0, 1400.0, "fallback"


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def shipping_inputs():
    fact = gen.fact_table(N_FACT, N_DIM, SEED2, cols=("key", "price", "disc", "date"))
    dim = gen.dim_table(N_DIM, SEED2, cols=("key", "segment"))
    return fact, dim


# --------------------------------------------------------------- CPU oracle

def _timed(fn):
    t0 = time.perf_counter()
    fn()
    return time.perf_counter() - t0


def cpu_shipping_sample(scale: int, parallel: bool):
    """The oracle on a 1/scale sample of the shipping-priority workload (same
    generator, key range scaled with it).  Returns (fact rows, seconds)."""
    from oracle import relational as R
    nf, nd = N_FACT // scale, N_DIM // scale
    fact = gen.fact_table(nf, nd, SEED2 + 1000 + scale, cols=("key", "price", "disc", "date"))
    dim = gen.dim_table(nd, SEED2 + 1000 + scale, cols=("key", "segment"))

    def q():
        bsel = R.filter([(dim["segment"], "==", 2)], nd, parallel=parallel)
        psel = R.filter([(fact["date"], ">", 1200)], nf, parallel=parallel)
        prow, _, _ = R.join(dim["key"], fact["key"], bsel=bsel, psel=psel, parallel=parallel)
        keys, aggs = R.groupby([fact["key"]], [("sum_mul_kminus", fact["price"], fact["disc"], 100)], nf, sel=prow,
                               parallel=parallel)
        R.topk(aggs[:, 0], keys[:, 0], 10)

    return nf, _timed(q)


def cpu_pricing_sample(scale: int, parallel: bool):
    from oracle import relational as R
    n = N_FACT // scale
    t = gen.fact_table(n, N_DIM // scale, SEED2 + 2000, cols=("flag", "status", "qty", "price", "disc", "date"))

    def q():
        sel = R.filter([(t["date"], "<=", 2460)], n, parallel=parallel)
        R.groupby([t["flag"], t["status"]], [("sum", t["qty"], None, None), ("sum", t["price"], None, None),
                                              ("sum_mul_kminus", t["price"], t["disc"], 100),
                                              ("count", None, None, None), ("avg", t["qty"], None, None)], n,
                  sel=sel, parallel=parallel)

    return n, _timed(q)


def cpu_filter_sample(scale: int, parallel: bool):
    from oracle import relational as R
    n = N_FACT // scale
    t = gen.fact_table(n, N_DIM // scale, SEED2 + 3000, cols=("date",))
    return n, _timed(lambda: R.filter([(t["date"], "<=", 2460)], n, parallel=parallel))


def cpu_chain_sample(scale: int, parallel: bool):
    from oracle import relational as R
    npr, nb, nt = 100_000_000 // scale, 10_000_000 // scale, 1_000_000 // scale
    d = gen.chain_tables(npr, nb, nt, gen.BASE_SEED + 2 + 1000 * scale)

    def q():
        b_rows, t_rows, _ = R.join(d["third_pk"], d["build_fk2"], cap=nb, parallel=parallel)
        cat_of = d["third_cat"][t_rows]
        p_rows, ib, _ = R.join(d["build_pk"][b_rows], d["probe_fk"].astype(np.int32), cap=npr, parallel=parallel)
        cat = np.ascontiguousarray(cat_of[ib], dtype=np.int32)
        pay = np.ascontiguousarray(d["probe_payload"][p_rows])
        R.groupby([cat], [("sum", pay, None, None), ("count", None, None, None)], len(cat), parallel=parallel)

    return npr, _timed(q)


def cpu_nm_sample(scale: int, parallel: bool):
    from oracle import relational as R
    nb, npr = 10_000_000 // scale, 20_000_000 // scale
    d = gen.nm_join_tables(nb, npr, 12.0, gen.BASE_SEED + 6 + 1000 * scale)

    def q():
        psel = R.filter([(d["probe_date"], ">", 1200)], npr, parallel=parallel)
        R.join(d["build_key"], d["probe_key"], psel=psel, parallel=parallel)

    return npr, _timed(q)


def cpu_soft_sample(n: int):
    """Soft aggregation forward + backward in float64 (numpy, one thread)."""
    from oracle import soft
    s = gen.soft_table(n, 1024, gen.BASE_SEED + 3)
    th = np.zeros(1024, np.float32)
    ones = np.ones(1024)

    def q():
        soft.soft_agg_fwd(s["x"], s["v"], s["gid"], th, 0.1, 1024)
        soft.soft_agg_bwd(s["x"], s["v"], s["gid"], th, 0.1, 1024, ones, ones)

    return n, _timed(q)


def cpu_cnn_sample(grids: int = 1):
    """One trainable-query step (forward, backward, Adam) of the float64 CNN
    oracle on `grids` grids of 16 cells."""
    from oracle import cnn as O
    img, lab = gen.glyph_grids(grids, gen.BASE_SEED + 4)
    params = {k: np.asarray(v, np.float64) for k, v in gen.cnn_params(gen.BASE_SEED + 5).items()}
    tgt = O.targets_from_labels(lab)
    zeros = {k: np.zeros_like(v) for k, v in params.items()}

    def q():
        fw = O.forward(params, img)
        g = O.backward(params, fw, tgt)
        O.adam_step(params, g, zeros, zeros, 1)

    return grids * 16, _timed(q)


def cpu_dict_sample(n: int = 1_000_000, parallel: bool = False):
    """Dictionary codes of n strings of the dictionary workload (the oracle:
    Python's sort of the distinct byte strings), then GROUP BY (code, flag)
    with the plain C oracle."""
    from oracle import dictionary as D
    from oracle import relational as R
    off, data, vocab, idx = gen.string_column(n, 100_000, gen.BASE_SEED + 7, max_len=24)
    flag = gen.fact_table(n, 1, gen.BASE_SEED + 7, cols=("flag", "price"))
    strs = D.split(off, data)
    out = {}

    def enc():
        out["codes"] = D.dict_encode(strs)[0]

    s_enc = _timed(enc)
    s_gb = _timed(lambda: R.groupby([out["codes"].astype(np.int64), flag["flag"]],
                                    [("sum", flag["price"], None, None), ("count", None, None, None)], n,
                                    parallel=parallel))
    return n, s_enc, s_gb


def cpu_soft_filter_sample(n: int = 1_000_000):
    """Soft filter forward + backward in float64 (numpy, one thread)."""
    from oracle import soft
    s = gen.soft_table(n, 1024, gen.BASE_SEED + 3)
    th = np.zeros(1024, np.float32)
    gm = np.ones(n)

    def q():
        soft.soft_filter_fwd(s["x"], s["gid"], th, 0.1)
        soft.soft_filter_bwd(s["x"], s["gid"], th, 0.1, 1024, gm)

    return n, _timed(q)


def cpu_pair_sample(grids: int = 1):
    """One Digit x Size query step (forward, backward, Adam) of the float64
    oracle on `grids` grids of 16 cells."""
    from oracle import cnn as O
    img, dig, siz = gen.glyph_grids_sized(grids, gen.BASE_SEED + 6)
    params = {k: np.asarray(v, np.float64) for k, v in gen.cnn_params(gen.BASE_SEED + 5).items()}
    sp = {k: np.asarray(v, np.float64) for k, v in gen.size_head_params(gen.BASE_SEED + 5).items()}
    tgt = O.targets2(dig, siz)
    allp = dict(params, **sp)
    zeros = {k: np.zeros_like(v) for k, v in allp.items()}

    def q():
        fw = O.forward2(params, sp, img)
        g = O.backward2(params, sp, fw, tgt)
        O.adam_step(allp, g, zeros, zeros, 1)

    return grids * 16, _timed(q)


def cpu_llp_sample(n: int = 1_000_000, B: int = 64):
    """One LLP training step (forward, backward, Adam) of the float64 oracle
    on n census-shaped rows in bags of B."""
    from oracle import cnn as O
    from oracle import llp as R
    X, y = gen.llp_table(n, gen.BASE_SEED + 9)
    t = R.bag_counts(y, B).astype(np.float64)
    p = {"W": np.zeros((2, 6)), "b": np.zeros(2)}
    z = {k: np.zeros_like(v) for k, v in p.items()}

    def q():
        fw = R.forward(X, p["W"], p["b"], B)
        O.adam_step(p, R.backward(X, fw, t, B), z, z, 1)

    return n, _timed(q)


def cpu_softsort_sample(groups: int = 20):
    """The float64 oracle's soft top-10 forward and backward on `groups` groups
    of the ranked-groups workload."""
    from oracle import softsort as O
    d = gen.ranked_groups(1000, 1000, gen.BASE_SEED + 11)
    offs = d["offsets"][:groups + 1]
    x, v = d["x"][:offs[-1]], d["v"][:offs[-1]]
    pairs = float(np.sum(np.diff(offs).astype(np.float64) ** 2))

    def q():
        _, m, _ = O.soft_topk_fwd(x, v, offs, 10, 0.05, 0.5)
        O.soft_topk_bwd(x, v, offs, 10, 0.05, 0.5, m, dS=np.ones(groups))

    return pairs, _timed(q)


# special-function (MUFU) results per SM per clock: 2^x and 1/x of a logistic
MUFU_PER_SM_CLK = 16


def cpu_baseline(fn, unit_scale: float, unit: str, sample: str, parallel_ok: bool = True, **kw):
    """Times the oracle: OpenMP on all host cores (when the function has a
    parallel form) and single-threaded.  Rates are units per second of
    `unit` (work per sample unit x unit_scale)."""
    from oracle import relational as R
    out = {"unit": unit, "kind": "oracle", "sample": sample}
    n1, s1 = fn(parallel=False, **kw) if parallel_ok else fn(**kw)
    out["single_thread"] = {"value": n1 * unit_scale / s1, "seconds": s1, "cores": 1}
    if parallel_ok:
        n2, s2 = fn(parallel=True, **kw)
        out.update({"value": n2 * unit_scale / s2, "seconds": s2, "cores": R.threads()})
    else:
        out.update({"value": out["single_thread"]["value"], "seconds": s1, "cores": 1})
    out["host_cores"] = host_cores()
    return out


def run_reference(args):
    """The reference arm: the oracle (plain C, OpenMP on the host cores) on a
    bounded sample of the headline workload, per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import relational as R
    scale = 20
    rows, secs = [], []
    for _ in range(args.warmup):
        cpu_shipping_sample(scale, True)
    for _ in range(args.steps):
        r, s = cpu_shipping_sample(scale, True)
        rows.append(r)
        secs.append(s)
    v = sum(rows) / sum(secs)
    line = {
        "impl": "reference", "metric": "fact rows/s (shipping-priority plan)", "value": v, "unit": "rows/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * sum(secs) / len(secs), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "fact_rows": N_FACT, "dim_rows": N_DIM,
                   "parallelism": "replicas" if args.gpus > 1 else "single-gpu"},
        "cpu_baseline": {"value": v, "unit": "rows/s", "cores": R.threads(), "host_cores": host_cores(),
                         "kind": "oracle",
                         "sample": "1/%d of the workload per step (%d fact rows, %d dimension rows), plain C "
                                   "oracle, OpenMP row-partitioned" % (scale, N_FACT // scale, N_DIM // scale)},
        "e2e": {"value": v, "unit": "rows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- traffic

# DRAM bytes (read + write) of a kernel per unit of its workload (fact rows,
# probe rows ...) from one ncu capture summarised in profiles/, with the
# source file it was built from (first 12 hex digits of its sha1).  Captures
# run a smaller case of the same plan; every term of these kernels' traffic
# grows with those units, so it is scaled by them.  None when the source
# changed since the capture.
TRAFFIC = {
    # gjr_probe_kernel at 1/4 scale (15M fact rows): 327.60 MB read + 3.19 MB written
    "gjr_probe": {"src": "paper_2211_02753_b300/csrc/groupjoin.cu", "sha1": "69c6b8e2ce61",
                  "bytes_per_unit": (327_599_616 + 3_187_456) / 15_000_000},
    # llp_stream_kernel<6, true> on 8M census-shaped rows (bags of 64): 193.25 MB read + 0.04 MB written
    "llp_stream": {"src": "paper_2211_02753_b300/csrc/llp.cu", "sha1": "254578b3f29e",
                   "bytes_per_unit": (193_246_720 + 37_632) / 8_000_000},
    # filter_kernel<4> on 60M rows (date <= 2460): 240.10 MB read + 170.58 MB written (the last
    # ~60 MB of row ids are still in L2 when the kernel ends)
    "filter": {"src": "paper_2211_02753_b300/csrc/filter.cu", "sha1": "6155f4a8d054",
               "bytes_per_unit": (240_095_744 + 170_581_248) / 60_000_000},
    # small_domain_priv_n_kernel<5, 1, 3> on 15M rows of the pricing summary: 450.07 MB read + 2.90 MB written
    "small_domain_priv": {"src": "paper_2211_02753_b300/csrc/groupby.cu", "sha1": "c3865440c0bb",
                          "bytes_per_unit": (450_068_992 + 2_904_064) / 15_000_000},
    # soft_reduce_kernel<0> / <1> on the 10M-row soft query: 120.18 MB read + 4.50 / 2.15 MB written
    "soft_reduce_fwd": {"src": "paper_2211_02753_b300/csrc/soft.cu", "sha1": "c1765360f92f",
                        "bytes_per_unit": (120_178_944 + 4_499_968) / 10_000_000},
    "soft_reduce_bwd": {"src": "paper_2211_02753_b300/csrc/soft.cu", "sha1": "c1765360f92f",
                        "bytes_per_unit": (120_182_016 + 2_154_240) / 10_000_000},
}


def measured_traffic(kernel: str, units: float):
    import hashlib
    t = TRAFFIC.get(kernel)
    if t is None:
        return None
    with open(os.path.join(ROOT, t["src"]), "rb") as f:
        if hashlib.sha1(f.read()).hexdigest()[:12] != t["sha1"]:
            return None
    return t["bytes_per_unit"] * units


def roofline(bound, algo, seconds, peak, unit, kernel, traffic=None, peak_kind="measured", extra=None):
    achieved = algo / seconds / (1e9 if unit == "GB/s" else 1e12)
    r = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
         "traffic": traffic, "kernel": kernel, "peak_kind": peak_kind,
         "algorithmic": algo, "seconds": seconds}
    if traffic is not None and unit == "GB/s":
        r["dram_gbs"] = traffic / seconds / 1e9
        r["dram_frac"] = r["dram_gbs"] / peak
    if extra:
        r.update(extra)
    return r


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

def _events_median(fns, stream, reps=5):
    """Median CUDA-event time (ms) of each function in `fns`, run in order on
    `stream` (each is a library call; events recorded between them).  A
    bounded ~1 ms device sleep is queued first, so that the host has issued
    every call before the GPU reaches the first event: the intervals then
    hold the calls' device time only, not the host's argument marshalling
    and launch latency (which the graph-replayed step does not pay)."""
    import torch
    ts = []
    for _ in range(reps):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(len(fns) + 1)]
        with torch.cuda.stream(stream):
            torch.cuda._sleep(2_000_000)
        e[0].record(stream)
        for i, fn in enumerate(fns):
            fn()
            e[i + 1].record(stream)
        torch.cuda.synchronize()
        ts.append([e[i].elapsed_time(e[i + 1]) for i in range(len(fns))])
    return [statistics.median(t[i] for t in ts) for i in range(len(fns))]


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

    hbm_peak, bf16_peak, peak_kind = load_peaks()

    # ---- headline: shipping-priority plan as one group-join
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

    # stage timing (CUDA events on the launching stream): build, probe, finish
    st_ms = _events_median([plan.gj_build, plan.gj_probe, plan.gj_finish], stream)
    ops.check(plan.status, "shipping-priority stages")

    # the timed step: the plan captured once as a CUDA graph and replayed
    # (the same kernels; no host work between launches)
    step = plans.Graphed(plan)
    out = step.run()
    torch.cuda.synchronize()
    ops.check(plan.status, "shipping-priority plan (graph)")
    assert int(out["nmatch"].item()) == nmatch and int(out["ngroups"].item()) == ngroups

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

    # ---- roofline of the dominant kernel: the probe (algorithmic bytes of
    # the fact side per the plan's byte budget: the date column, the key of
    # every row passing date > 1200, price and discount of every match;
    # bitmap lookups and accumulator atomics are L2-resident and not counted)
    sel_f = float(np.mean(fact_h["date"] > 1200))
    probe_algo = N_FACT * 4 + N_FACT * sel_f * 4 + nmatch * 16
    build_algo = N_DIM * 1 + N_DIM * 0.2 * 4
    finish_algo = ngroups * 12
    stage_names = ["groupjoin_build", "groupjoin_probe", "groupjoin_finish"]
    roof = roofline("hbm", probe_algo, st_ms[1] / 1e3, hbm_peak, "GB/s", "gjr_probe_kernel (tdp_groupjoin_probe)",
                    traffic=measured_traffic("gjr_probe", N_FACT), peak_kind=peak_kind + " (copy bandwidth)",
                    extra={"stages_ms": dict(zip(stage_names, st_ms)),
                           "stages_algo_gbs": {n: a / (t / 1e3) / 1e9 for n, a, t in
                                               zip(stage_names, [build_algo, probe_algo, finish_algo], st_ms)},
                           "plan_algorithmic_bytes": build_algo + probe_algo + finish_algo,
                           "plan_frac": (build_algo + probe_algo + finish_algo) / (ms / 1e3) / 1e9 / hbm_peak})

    line = {
        "metric": "fact rows/s (shipping-priority plan)", "value": value, "unit": "rows/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "fact_rows": N_FACT, "dim_rows": N_DIM, "matches": nmatch,
                   "groups": ngroups, "parallelism": "replicas" if world > 1 else "single-gpu",
                   "plan": "group-join (build / probe / finish) with fused top-10",
                   "l2": "inputs larger than L2 (1.5 GB of columns per step)",
                   "launch": "each step one replay of the plan captured as a CUDA graph"},
        "roofline": roof,
        "e2e": {"value": e2e_value, "unit": "rows/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e2e_ms},
        "gpu_launches": (launches_per_step * args.steps) if launches_per_step is not None else None,
        "gpu_launches_per_step": launches_per_step,
        "clocks": clocks,
    }
    del fact, dim, plan, step, pin_f, pin_d
    torch.cuda.empty_cache()

    if args.plans == "all":
        line["plans"] = other_plans(dev, stream, hbm_peak, bf16_peak, peak_kind, args, fact_h, dim_h)

    if rank == 0:
        scale = 20
        line["cpu_baseline"] = cpu_baseline(
            cpu_shipping_sample, 1.0, "rows/s",
            "1/%d of the workload (%d fact rows, %d dimension rows), plain C oracle" %
            (scale, N_FACT // scale, N_DIM // scale), scale=scale)
        for name in ("shipping_separate_partition", "shipping_separate_sort"):
            if name in line.get("plans", {}):
                line["plans"][name]["cpu_baseline"] = dict(line["cpu_baseline"],
                                                           note="the same query's oracle as the headline")
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


def other_plans(dev, stream, hbm_peak, bf16_peak, peak_kind, args, fact_h, dim_h):
    import torch
    from paper_2211_02753_b300 import ops, plans
    res = {}
    steps = max(3, min(args.steps, 50))
    pk = peak_kind + " (copy bandwidth)"
    # ---- shipping priority on the separate path (build -> probe -> group-by -> top-k)
    fact = {k: torch.from_numpy(v).to(dev) for k, v in fact_h.items()}
    dim = {k: torch.from_numpy(v).to(dev) for k, v in dim_h.items()}
    sel_f = float(np.mean(fact_h["date"] > 1200))
    for strategy in ("auto", "sort"):
        p = plans.ShippingPriority(fact, dim, groupjoin=False, groupby_strategy=strategy)
        ms = _time_graph(lambda: p.run(), stream, steps)
        o = p.run()
        torch.cuda.synchronize()
        ops.check(p.status, "shipping separate " + strategy)
        nm, ng = int(o["nmatch"].item()), int(o["ngroups"].item())
        # the group-by stage on its own (CUDA events): 12 B/match scattered or
        # sorted (3 digit passes x 2 x 12 B for the sort path) + groups out
        kc, pc, dc = p.last_probe["gathered"]
        gb_ms = _events_median([lambda: ops.groupby_agg([ops.Col(kc, 1, N_DIM), pc, dc], [0],
                                                        [("sum_mul_kminus", 1, 2, 100)], n=p.cap,
                                                        nsel=p.last_probe["count"], strategy=strategy,
                                                        capacity=p.cap, status=p.status)], stream)[0]
        gb_algo = nm * 20 + (nm * 12 * 2 * 3 if strategy == "sort" else nm * 24) + ng * 12
        res["shipping_separate_" + ("partition" if strategy == "auto" else "sort")] = {
            "ms": ms, "rows_per_s": N_FACT / (ms / 1e3), "groups": ng, "groupby_ms": gb_ms,
            "roofline": roofline("hbm", gb_algo, gb_ms / 1e3, hbm_peak, "GB/s", "group-by stage (" + strategy + ")",
                                 peak_kind=pk)}
        del p
        torch.cuda.empty_cache()
    del fact, dim
    torch.cuda.empty_cache()
    # ---- filter and pricing summary at 60M rows
    t = gen.fact_table(N_FACT, N_DIM, SEED2, cols=("flag", "status", "qty", "price", "disc", "date"))
    sel = float(np.mean(t["date"] <= 2460))
    td = {k: torch.from_numpy(v).to(dev) for k, v in t.items()}
    del t
    fout = {}

    def run_filter():
        fout["o"] = ops.filter([td["date"]], [(0, "<=", 2460)], rowids=True)

    ms = _time_graph(run_filter, stream, steps)
    nsel = int(fout["o"]["count"].item())
    fbytes = N_FACT * 4 + nsel * 4
    res["filter_60M"] = {"ms": ms, "rows_per_s": N_FACT / (ms / 1e3), "selected": nsel,
                         "roofline": roofline("hbm", fbytes, ms / 1e3, hbm_peak, "GB/s", "filter_kernel",
                                              traffic=measured_traffic("filter", N_FACT), peak_kind=pk),
                         "cpu_baseline": cpu_baseline(cpu_filter_sample, 1.0, "rows/s",
                                                      "1/10 of the rows (6M), date <= 2460", scale=10)}
    for strategy in ("small_domain", "sort"):
        p = plans.PricingSummary(td, strategy)
        ms = _time_graph(lambda: p.run(), stream, steps if strategy == "small_domain" else 3)
        algo = N_FACT * plans.PricingSummary.bytes_per_row(sel)
        if strategy == "sort":  # plus the pack and the sort passes over (key, row) pairs of the selected rows
            algo += N_FACT * sel * (12 + 2 * 12)
        res["pricing_summary_60M_" + strategy] = {
            "ms": ms, "rows_per_s": N_FACT / (ms / 1e3),
            "roofline": roofline("hbm", algo, ms / 1e3, hbm_peak, "GB/s",
                                 "small_domain_priv_n_kernel" if strategy == "small_domain" else "sort path",
                                 traffic=measured_traffic("small_domain_priv", N_FACT)
                                 if strategy == "small_domain" else None, peak_kind=pk)}
    res["pricing_summary_60M_small_domain"]["cpu_baseline"] = cpu_baseline(
        cpu_pricing_sample, 1.0, "rows/s", "1/20 of the rows (3M)", scale=20)
    del td
    torch.cuda.empty_cache()
    # ---- join chain (100M probe rows): fused, and probe -> sort group-by
    d = gen.chain_tables(100_000_000, 10_000_000, 1_000_000, gen.BASE_SEED + 2)
    dd = {k: torch.from_numpy(v.astype(np.int32) if k == "probe_fk" else v).to(dev) for k, v in d.items()}
    del d
    for name, fused, strategy in (("join_chain_100M", True, "auto"), ("join_chain_100M_sort", False, "sort")):
        jc = plans.JoinChain(dd, fused=fused, groupby_strategy=strategy)
        ms = _time_graph(lambda: jc.run(), stream, steps if fused else 3)
        out = jc.run()
        torch.cuda.synchronize()
        ops.check(jc.status, name)
        # probe 12 B/row (key + payload), build 10M x (4 + 4 + 8 slot), third 1M x 8, tables written;
        # the unfused path adds 12 B/match written + the sort (2 x 12 B x 3 passes) + read back
        algo = 100e6 * 12 + 10e6 * (4 + 4 + 8 + 8) + 1e6 * 8 + 2 ** 24 * 8 + 2 ** 21 * 8
        if not fused:
            algo += 100e6 * (12 + 12 * 2 * 3 + 12)
        res[name] = {"ms": ms, "rows_per_s": 100e6 / (ms / 1e3), "groups": int(out["ngroups"].item()),
                     "roofline": roofline("hbm", algo, ms / 1e3, hbm_peak, "GB/s",
                                          "join_probe_agg_kernel" if fused else "probe + sort group-by",
                                          peak_kind=pk)}
        del jc, out
        torch.cuda.empty_cache()
    res["join_chain_100M"]["cpu_baseline"] = cpu_baseline(cpu_chain_sample, 1.0, "rows/s",
                                                          "1/50 of the chain (2M probe rows)", scale=50)
    del dd
    torch.cuda.empty_cache()
    # ---- N:M join: 10M build rows, about 12 per key; 20M probe rows, half of
    # the keys present, date > 1200 (~53%)
    d = gen.nm_join_tables(10_000_000, 20_000_000, 12.0, gen.BASE_SEED + 6)
    dd = {k: torch.from_numpy(v).to(dev) for k, v in d.items()}
    jn = {}

    def run_nm():
        jn["o"] = ops.join_nm([dd["build_key"]], 0, [dd["probe_key"], dd["probe_date"]], 0,
                              probe_preds=[(1, ">", 1200)], capacity=80_000_000)

    ms = _time_graph(run_nm, stream, min(steps, 10))
    pairs = int(jn["o"]["count"].item())
    ops.check(jn["o"]["status"], "join_nm")
    # build: key 4 B read, (key, row) 8 B written, 4 radix passes x 2 x 8 B, runs 8 B;
    # probe: key + date 8 B per row, 8 B per pair written
    algo = 10e6 * (4 + 8 + 4 * 16 + 8) + 20e6 * 8 + pairs * 8
    res["join_nm_10M_x_20M"] = {
        "ms": ms, "rows_per_s": 20e6 / (ms / 1e3), "pairs": pairs,
        "roofline": roofline("hbm", algo, ms / 1e3, hbm_peak, "GB/s", "N:M join (sort build + probe)", peak_kind=pk),
        "cpu_baseline": cpu_baseline(cpu_nm_sample, 1.0, "probe rows/s", "1/20 of both tables", scale=20)}
    del dd, jn
    torch.cuda.empty_cache()
    # ---- dictionary codes of a 10M-row string column (100k words, up to 24
    # bytes), then GROUP BY (code, flag)
    off, data, vocab, idx = gen.string_column(10_000_000, 100_000, gen.BASE_SEED + 7, max_len=24)
    flag = gen.fact_table(10_000_000, 1, gen.BASE_SEED + 7, cols=("flag", "price"))
    doff, ddat = torch.from_numpy(off).to(dev), torch.from_numpy(data).to(dev)
    fl, pr = torch.from_numpy(flag["flag"]).to(dev), torch.from_numpy(flag["price"]).to(dev)
    enc = {}

    def run_enc():
        enc["o"] = ops.dict_encode(doff, ddat, max_len=24)

    ms = _time_graph(run_enc, stream, min(steps, 10))
    ops.check(enc["o"]["status"], "dict_encode")
    nd = int(enc["o"]["ndict"].item())
    algo = data.nbytes + off.nbytes + 10e6 * 4
    res["dict_encode_10M"] = {
        "ms": ms, "rows_per_s": 10e6 / (ms / 1e3), "distinct": nd,
        "roofline": roofline("hbm", algo, ms / 1e3, hbm_peak, "GB/s",
                             "dictionary encoding (hash dedup of the rows, sort of the distinct strings)",
                             peak_kind=pk,
                             extra={"note": "algorithmic = strings + offsets read, codes written; the words "
                                            "(28 B per row) are written and read back, and the distinct "
                                            "strings take 25 digit passes on top"})}
    codes = enc["o"]["codes"]
    gcols = [ops.Col(codes, 0, nd - 1), ops.Col(fl, 0, 2), pr]
    ms = _time_graph(lambda: ops.groupby_agg(gcols, [0, 1], [("sum", 2), ("count",)], capacity=3 * nd), stream,
                     min(steps, 10))
    res["dict_groupby_10M"] = {
        "ms": ms, "rows_per_s": 10e6 / (ms / 1e3),
        "roofline": roofline("hbm", 10e6 * (4 + 1 + 8), ms / 1e3, hbm_peak, "GB/s",
                             "GROUP BY (dictionary code, flag)", peak_kind=pk)}
    n1, s_enc, s_gb = cpu_dict_sample()
    res["dict_encode_10M"]["cpu_baseline"] = {
        "value": n1 / s_enc, "unit": "strings/s", "cores": 1, "kind": "oracle", "host_cores": host_cores(),
        "sample": "1M strings of the same column: the oracle's sort of the distinct byte strings (%.2f s)" % s_enc}
    res["dict_groupby_10M"]["cpu_baseline"] = {
        "value": n1 / s_gb, "unit": "rows/s", "cores": 1, "kind": "oracle", "host_cores": host_cores(),
        "sample": "1M rows: the plain C oracle's GROUP BY (code, flag), one thread (%.2f s)" % s_gb}
    del doff, ddat, fl, pr, enc, codes, gcols
    torch.cuda.empty_cache()
    # ---- soft query (10M rows)
    s = gen.soft_table(10_000_000, 1024, gen.BASE_SEED + 3)
    sd = {k: torch.from_numpy(v).to(dev) for k, v in s.items()}
    sq = plans.SoftQuery(sd)
    ms = _time_graph(lambda: sq.run(), stream, steps)
    res["soft_query_10M_fwd_bwd"] = {
        "ms": ms, "rows_per_s": 10e6 / (ms / 1e3),
        "roofline": roofline("hbm", 10e6 * 24, ms / 1e3, hbm_peak, "GB/s", "soft_reduce_kernel fwd + bwd",
                             peak_kind=pk),
        "cpu_baseline": cpu_baseline(cpu_soft_sample, 1.0, "rows/s", "1M rows, float64 numpy, one thread",
                                     parallel_ok=False, n=1_000_000)}
    th, tau = sq.theta, sq.tau
    gm = torch.ones_like(sd["x"])
    for name, fn, bpr, kern, tkey in (
            ("soft_agg_fwd_10M", lambda: ops.soft_agg_fwd(sd["x"], sd["v"], sd["gid"], th, tau), 12,
             "soft_reduce_kernel<fwd>", "soft_reduce_fwd"),
            ("soft_agg_bwd_10M", lambda: ops.soft_agg_bwd(sd["x"], sd["v"], sd["gid"], th, tau, sq.gS, sq.gC), 12,
             "soft_reduce_kernel<bwd>", "soft_reduce_bwd"),
            ("soft_filter_fwd_10M", lambda: ops.soft_filter_fwd(sd["x"], sd["gid"], th, tau), 12,
             "soft_filter_fwd_kernel", None),
            ("soft_filter_bwd_10M", lambda: ops.soft_filter_bwd(sd["x"], sd["gid"], th, tau, gm), 16,
             "soft_reduce_kernel<filter bwd>", None)):
        ms = _time_graph(fn, stream, steps)
        res[name] = {"ms": ms, "rows_per_s": 10e6 / (ms / 1e3),
                     "roofline": roofline("hbm", 10e6 * bpr, ms / 1e3, hbm_peak, "GB/s", kern,
                                          traffic=measured_traffic(tkey, 10e6) if tkey else None, peak_kind=pk)}
    n1, s1 = cpu_soft_filter_sample()
    sfb = {"value": n1 / s1, "unit": "rows/s", "cores": 1, "kind": "oracle", "host_cores": host_cores(),
           "sample": "1M rows, soft filter forward + backward, float64 numpy, one thread (%.2f s)" % s1}
    res["soft_filter_fwd_10M"]["cpu_baseline"] = sfb
    res["soft_filter_bwd_10M"]["cpu_baseline"] = sfb
    for name in ("soft_agg_fwd_10M", "soft_agg_bwd_10M"):
        res[name]["cpu_baseline"] = dict(res["soft_query_10M_fwd_bwd"]["cpu_baseline"],
                                         note="the oracle's soft aggregation forward + backward")
    # variants of one query share its oracle timing (the oracle has no strategies)
    for name, base in (("pricing_summary_60M_sort", "pricing_summary_60M_small_domain"),
                       ("join_chain_100M_sort", "join_chain_100M")):
        res[name]["cpu_baseline"] = dict(res[base]["cpu_baseline"], note="the same query's oracle as " + base)
    del sd, sq
    torch.cuda.empty_cache()
    res["trainable_query_glyph_cnn"] = glyph_plan(dev, stream, args, bf16_peak, peak_kind)
    res["trainable_query_digit_x_size"] = pair_plan(dev, stream, args, bf16_peak, peak_kind)
    res.update(llp_plans(dev, stream, args, hbm_peak, peak_kind))
    res["soft_topk_1000_groups"] = softsort_plan(dev, stream, args)
    return res


def glyph_plan(dev, stream, args, bf16_peak, peak_kind):
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
    train_flops = 3 * flops_fwd
    cells, secs = cpu_cnn_sample(1)
    return {"train_ms": train_ms, "train_steps_per_s": 1000.0 / train_ms, "exact_query_ms": infer_ms,
            "exact_query_steps_per_s": 1000.0 / infer_ms, "batch_grids": B, "training_steps": budget,
            "query_accuracy": float(ok.mean()), "cell_accuracy": cell_acc,
            "roofline": roofline("tensor", train_flops, train_ms / 1e3, bf16_peak, "TFLOP/s",
                                 "whole training step (conv2 tcgen05 kernels, fc1 tcgen05 GEMM)",
                                 peak_kind=peak_kind + " (cuBLAS bf16, sustained)"),
            "cpu_baseline": {"value": 1.0 / (secs * 4096 / cells), "unit": "train steps/s", "cores": 1,
                             "kind": "oracle", "host_cores": host_cores(),
                             "sample": "one grid (16 cells) through the float64 oracle's forward, backward and "
                                       "Adam (%.2f s), scaled per cell to the 4096-cell step" % secs}}


def pair_plan(dev, stream, args, bf16_peak, peak_kind):
    """The Digit x Size trainable query (two heads, soft pair COUNT): train
    steps/s at batch 256 grids, exact pair-query steps/s, and the exact pair
    query's accuracy on 1024 held-out grids after a fixed training budget."""
    import torch
    from oracle import cnn as O  # targets: the exact pair counts on the true labels
    from oracle import soft
    from paper_2211_02753_b300 import cnn
    tr_img, tr_dig, tr_siz = gen.glyph_grids_sized(4096, gen.BASE_SEED + 6)
    te_img, te_dig, te_siz = gen.glyph_grids_sized(1024, gen.BASE_SEED + 106)
    targets = torch.from_numpy(O.targets2(tr_dig, tr_siz).astype(np.float32)).to(dev)
    g_tr = torch.from_numpy(tr_img).to(dev)
    g_te = torch.from_numpy(te_img).to(dev)
    q = cnn.GlyphQuery2(gen.cnn_params(gen.BASE_SEED + 5), gen.size_head_params(gen.BASE_SEED + 5), dev, lr=1e-3,
                        warmup=400)
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
    budget = 2400
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
    ld, ls, cnt = q.exact_query(g_te)
    e = soft.exact_groupby2(te_dig, te_siz).reshape(1024, -1)
    ok = np.all(cnt.cpu().numpy().reshape(1024, -1) == e, axis=1)
    flops_fwd = 4096 * 2 * (26 * 26 * 32 * 9 + 24 * 24 * 64 * 288 + 9216 * 128 + 128 * 12)
    cells, secs = cpu_pair_sample(1)
    return {"train_ms": train_ms, "train_steps_per_s": 1000.0 / train_ms, "exact_query_ms": infer_ms,
            "exact_query_steps_per_s": 1000.0 / infer_ms, "batch_grids": B, "training_steps": budget,
            "pair_query_accuracy": float(ok.mean()),
            "digit_cell_accuracy": float((ld.cpu().numpy().reshape(-1, 4, 4) == te_dig).mean()),
            "size_cell_accuracy": float((ls.cpu().numpy().reshape(-1, 4, 4) == te_siz).mean()),
            "roofline": roofline("tensor", 3 * flops_fwd, train_ms / 1e3, bf16_peak, "TFLOP/s",
                                 "whole training step (conv2 tcgen05 kernels, fc1 tcgen05 GEMM)",
                                 peak_kind=peak_kind + " (cuBLAS bf16, sustained)"),
            "cpu_baseline": {"value": 1.0 / (secs * 4096 / cells), "unit": "train steps/s", "cores": 1,
                             "kind": "oracle", "host_cores": host_cores(),
                             "sample": "one grid (16 cells) through the float64 oracle's two-head forward, "
                                       "backward and Adam (%.2f s), scaled per cell to the 4096-cell step" % secs}}


LLP_ROWS = 64_000_000
LLP_BAG = 64


def llp_plans(dev, stream, args, hbm_peak, peak_kind):
    """Learning from label proportions: (1) training throughput on 64M
    census-shaped rows (6 fp32 features, bags of 64, label-DP counts at
    eps = 0.1), one full-batch step = the fused forward + backward pass and
    Adam; (2) the paper's experiment on census-sized data (32,561 training
    rows, 16,281 test rows): test error after 300 steps per bag size, with
    exact and with Laplace counts, and the step time at that size."""
    import torch
    from oracle import llp as R  # count labels of the throughput workload
    from paper_2211_02753_b300 import llp
    out = {}
    X, y = gen.llp_table(LLP_ROWS, gen.BASE_SEED + 9)
    gX, gy = torch.from_numpy(X).to(dev), torch.from_numpy(y).to(dev)
    nb = R.n_bags(LLP_ROWS, LLP_BAG)
    noise = torch.from_numpy(gen.laplace_noise(nb, 2, gen.BASE_SEED + 10)).to(dev)
    del X, y
    t = llp.counts(gy, LLP_BAG, 2, noise=noise, eps=0.1)
    tr = llp.LLPTrainer(gX, t, LLP_BAG, np.zeros((2, 6)), np.zeros(2), lr=0.05)
    for _ in range(3):
        tr.step()
    n_timed = max(10, min(args.steps, 100))
    fb_ms, = _events_median([tr.forward_backward], stream, reps=n_timed)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(n_timed):
        tr.step()
    b.record(stream)
    torch.cuda.synchronize()
    step_ms = a.elapsed_time(b) / n_timed
    cnt_ms, = _events_median([lambda: llp.counts(gy, LLP_BAG, 2, noise=noise, eps=0.1)], stream, reps=10)
    algo = LLP_ROWS * 6 * 4 + nb * 2 * 4  # X once, the count labels once
    n1, s1 = cpu_llp_sample()
    out["llp_64M_bag64_dp"] = {
        "rows": LLP_ROWS, "features": 6, "bag": LLP_BAG, "eps": 0.1, "step_ms": step_ms,
        "rows_per_s": LLP_ROWS / (step_ms / 1e3), "forward_backward_ms": fb_ms, "dp_counts_ms": cnt_ms,
        "roofline": roofline("hbm", algo, fb_ms / 1e3, hbm_peak, "GB/s", "llp_stream_kernel + llp_reduce_kernel",
                             traffic=measured_traffic("llp_stream", LLP_ROWS), peak_kind=peak_kind),
        "cpu_baseline": {"value": n1 / s1, "unit": "rows/s", "cores": 1, "kind": "oracle",
                         "host_cores": host_cores(),
                         "sample": "one training step of the float64 oracle on 1M rows (%.2f s)" % s1}}
    del tr, gX, gy, noise, t
    torch.cuda.empty_cache()
    # ---- the paper's experiment at census size
    Xtr, ytr = gen.llp_table(32561, gen.BASE_SEED + 7)
    Xte, yte = gen.llp_table(16281, gen.BASE_SEED + 107)
    gtr, gytr = torch.from_numpy(Xtr).to(dev), torch.from_numpy(ytr).to(dev)
    gte, gyte = torch.from_numpy(Xte).to(dev), torch.from_numpy(yte).to(dev)
    table = {}
    small_ms = None
    for B in (1, 8, 16, 32, 64, 128, 256, 512):
        row = {}
        for dp in (False, True):
            nz = torch.from_numpy(gen.laplace_noise(R.n_bags(32561, B), 2, gen.BASE_SEED + 8)).to(dev) if dp \
                else None
            tt = llp.counts(gytr, B, 2, noise=nz, eps=0.1 if dp else None)
            tr = llp.LLPTrainer(gtr, tt, B, np.zeros((2, 6)), np.zeros(2), lr=0.05)
            a.record(stream)
            for _ in range(300):
                tr.step()
            b.record(stream)
            _, err = llp.predict(gte, tr.W, tr.b, gyte)
            row["llp_dp_error" if dp else "llp_error"] = int(err.item()) / len(yte)
            if B == 64 and not dp:
                small_ms = a.elapsed_time(b) / 300
        table[str(B)] = row
    out["llp_census_error_by_bag"] = {
        "train_rows": 32561, "test_rows": 16281, "steps": 300, "lr": 0.05, "eps": 0.1,
        "majority_class_error": float(np.mean(yte != 0)), "errors": table,
        "step_ms_at_bag_64": small_ms}
    return out


def softsort_plan(dev, stream, args):
    """Soft ORDER BY x DESC LIMIT 10 per group with the soft top-10 SUM of a
    payload: 1000 groups of 500..1500 rows (1.01M rows, 1.08e9 ordered
    pairs), forward + backward (dS = 1), and the exact operator."""
    import torch
    from paper_2211_02753_b300 import softsort as ss
    d = gen.ranked_groups(1000, 1000, gen.BASE_SEED + 11)
    gx, gv, go = (torch.from_numpy(d[k]).to(dev) for k in ("x", "v", "offsets"))
    pairs = float(np.sum(np.diff(d["offsets"]).astype(np.float64) ** 2))
    k, tau, tau_r, mg = 10, 0.05, 0.5, 1500
    dS = torch.ones(1000, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    fwd = lambda: ss.soft_topk_fwd(gx, gv, go, k, tau, tau_r, max_group=mg, status=st)  # noqa: E731
    _, mask, _ = fwd()
    bwd = lambda: ss.soft_topk_bwd(gx, gv, go, k, tau, tau_r, mask, dsum=dS, max_group=mg, status=st)  # noqa: E731
    exact = lambda: ss.exact_topk(gx, gv, go, k, max_group=mg, status=st)  # noqa: E731
    for _ in range(3):
        fwd(), bwd(), exact()
    reps = max(5, min(args.steps, 30))
    f_ms, b_ms, e_ms = _events_median([fwd, bwd, exact], stream, reps=reps)
    if int(st.item()) != 0:
        raise RuntimeError("soft top-k status %d" % int(st.item()))
    peak = MUFU_PER_SM_CLK * 148 * 2.032e9 / 1e12  # T special-function results / s
    n1, s1 = cpu_softsort_sample()
    ms = f_ms + b_ms
    return {"rows": int(d["offsets"][-1]), "groups": 1000, "pairs": pairs, "k": k, "tau": tau, "tau_r": tau_r,
            "fwd_ms": f_ms, "bwd_ms": b_ms, "exact_ms": e_ms, "pairs_per_s": pairs / (ms / 1e3),
            "roofline": {"bound": "alu", "achieved": 4 * pairs / (ms / 1e3) / 1e12, "peak": peak,
                         "unit": "T special-function results/s", "frac": 4 * pairs / (ms / 1e3) / 1e12 / peak,
                         "traffic": None, "kernel": "ss_rank_kernel<0> + ss_bwd_pair_kernel (2^x and 1/x, "
                                                    "2 per pair each)",
                         "peak_kind": "derived: 16 results per SM per clock x 148 SMs x 2032 MHz"},
            "cpu_baseline": {"value": n1 / s1, "unit": "pairs/s (forward + backward)", "cores": 1, "kind": "oracle",
                             "host_cores": host_cores(),
                             "sample": "20 groups (%.2e pairs) through the float64 oracle (%.2f s)" % (n1, s1)}}


def run_only(args):
    """One plan at 1/scale of its size, `steps` times after `warmup` runs, and
    a one-line timing (CUDA events).  Used for profiler captures of a small
    case; not the benchmark line."""
    import torch
    from paper_2211_02753_b300 import cnn, ops, plans
    from oracle import cnn as O  # glyph targets: the exact query on true labels
    dev = torch.device("cuda", 0)
    sc = max(1, args.scale)
    if args.only in ("shipping", "shipping_sep", "shipping_sort"):
        f, d = (gen.fact_table(N_FACT // sc, N_DIM // sc, SEED2, cols=("key", "price", "disc", "date")),
                gen.dim_table(N_DIM // sc, SEED2, cols=("key", "segment")))
        p = plans.ShippingPriority({k: torch.from_numpy(v).to(dev) for k, v in f.items()},
                                   {k: torch.from_numpy(v).to(dev) for k, v in d.items()},
                                   groupjoin=args.only == "shipping",
                                   groupby_strategy="sort" if args.only == "shipping_sort" else "auto")
        fn = p.run
    elif args.only in ("pricing", "pricing_sort", "filter"):
        t = gen.fact_table(N_FACT // sc, N_DIM // sc, SEED2, cols=("flag", "status", "qty", "price", "disc", "date"))
        td = {k: torch.from_numpy(v).to(dev) for k, v in t.items()}
        if args.only == "filter":
            fn = lambda: ops.filter([td["date"]], [(0, "<=", 2460)])  # noqa: E731
        else:
            fn = plans.PricingSummary(td, "sort" if args.only == "pricing_sort" else "small_domain").run
    elif args.only in ("chain", "chain_sort"):
        dd = gen.chain_tables(100_000_000 // sc, 10_000_000 // sc, 1_000_000 // sc, gen.BASE_SEED + 2)
        srt = args.only == "chain_sort"
        fn = plans.JoinChain({k: torch.from_numpy(v.astype(np.int32) if k == "probe_fk" else v).to(dev)
                              for k, v in dd.items()}, fused=not srt,
                             groupby_strategy="sort" if srt else "auto").run
    elif args.only == "soft":
        s = gen.soft_table(10_000_000 // sc, 1024, gen.BASE_SEED + 3)
        fn = plans.SoftQuery({k: torch.from_numpy(v).to(dev) for k, v in s.items()}).run
    elif args.only == "nm":
        d = gen.nm_join_tables(10_000_000 // sc, 20_000_000 // sc, 12.0, gen.BASE_SEED + 6)
        dd = {k: torch.from_numpy(v).to(dev) for k, v in d.items()}
        fn = lambda: ops.join_nm([dd["build_key"]], 0, [dd["probe_key"], dd["probe_date"]], 0,  # noqa: E731
                                 probe_preds=[(1, ">", 1200)], capacity=80_000_000 // sc)
    elif args.only in ("dict", "dict_groupby"):
        off, data, _, _ = gen.string_column(10_000_000 // sc, 100_000 // sc, gen.BASE_SEED + 7, max_len=24)
        doff, ddat = torch.from_numpy(off).to(dev), torch.from_numpy(data).to(dev)
        fn = lambda: ops.dict_encode(doff, ddat, max_len=24)  # noqa: E731
        if args.only == "dict_groupby":
            enc = fn()
            nd = int(enc["ndict"].item())
            flag = gen.fact_table(10_000_000 // sc, 1, gen.BASE_SEED + 7, cols=("flag", "price"))
            fl, pr = torch.from_numpy(flag["flag"]).to(dev), torch.from_numpy(flag["price"]).to(dev)
            gcols = [ops.Col(enc["codes"], 0, nd - 1), ops.Col(fl, 0, 2), pr]
            fn = lambda: ops.groupby_agg(gcols, [0, 1], [("sum", 2), ("count",)], capacity=3 * nd)  # noqa: E731
    elif args.only == "softsort":
        from paper_2211_02753_b300 import softsort as ss
        d = gen.ranked_groups(1000 // sc, 1000, gen.BASE_SEED + 11)
        gx, gv, go = (torch.from_numpy(d[k]).to(dev) for k in ("x", "v", "offsets"))
        _, mask, _ = ss.soft_topk_fwd(gx, gv, go, 10, 0.05, 0.5, max_group=1500)
        dS = torch.ones(1000 // sc, device=dev)

        def fn():
            ss.soft_topk_fwd(gx, gv, go, 10, 0.05, 0.5, max_group=1500)
            ss.soft_topk_bwd(gx, gv, go, 10, 0.05, 0.5, mask, dsum=dS, max_group=1500)
    elif args.only == "llp":
        from oracle import llp as R  # count labels of the workload
        from paper_2211_02753_b300 import llp
        n = LLP_ROWS // sc
        X, y = gen.llp_table(n, gen.BASE_SEED + 9)
        t = torch.from_numpy(R.bag_counts(y, LLP_BAG).astype(np.float32)).to(dev)
        tr = llp.LLPTrainer(torch.from_numpy(X).to(dev), t, LLP_BAG, np.zeros((2, 6)), np.zeros(2))
        fn = tr.forward_backward
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
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--plans", default="all", choices=["all", "main"])
    ap.add_argument("--only", default=None,
                    choices=["shipping", "shipping_sep", "shipping_sort", "pricing", "pricing_sort", "filter", "chain",
                             "chain_sort", "soft", "dict", "dict_groupby", "nm",
                             "glyph", "llp", "softsort"],
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
