"""Query plans of the benchmark workloads, composed from C-ABI calls.

Every plan runs on the current CUDA stream without a host synchronisation:
intermediate row counts stay on the device and flow into the next operator
through its d_n / d_nsel argument; capacities are host-side upper bounds.
A plan object owns its device buffers so that repeated steps allocate
nothing.

  PricingSummary  -- filter + group-by on the line-item table
                     (WHERE date <= 2460 GROUP BY flag, status: SUM qty,
                     SUM price, SUM price*(100-disc), COUNT, AVG qty)
  ShippingPriority -- dimension filter (segment = 2), fact filter (date >
                     1200), join on key, GROUP BY key SUM(price*(100-disc)),
                     top-10: one group-join call (default), or hash build ->
                     probe with a gather of key/price/disc -> group-by
  JoinChain       -- third (pk -> category) build; build rows probe it with
                     fk2 (category per build row); build (pk -> category);
                     probe rows probe it and aggregate SUM(payload), COUNT(*)
                     per category (fused probe + group-by)
  SoftQuery       -- soft filter + soft SUM/COUNT per group, forward and
                     backward (the trainable query of Sec. 4)
"""
from __future__ import annotations

import torch

from . import ops


class PricingSummary:
    def __init__(self, t: dict, strategy: str = "small_domain"):
        self.t = t  # key, flag, status, qty, price, disc, date (device tensors)
        self.cols = [t["flag"], t["status"], t["qty"], t["price"], t["disc"], t["date"]]
        self.cols[0] = ops.Col(t["flag"], 0, 2)
        self.cols[1] = ops.Col(t["status"], 0, 1)
        self.strategy = strategy
        self.aggs = [("sum", 2), ("sum", 3), ("sum_mul_kminus", 3, 4, 100), ("count",), ("avg", 2)]

    def run(self, status=None):
        return ops.groupby_agg(self.cols, [0, 1], self.aggs, preds=[(5, "<=", 2460)], strategy=self.strategy,
                               capacity=64, status=status)

    @staticmethod
    def bytes_per_row(selectivity: float) -> float:
        # date (4 B) always; flag, status (1+1 B), qty, price, disc (3x8 B) for
        # qualifying rows
        return 4.0 + selectivity * 26.0


class Graphed:
    """One step of a plan captured as a CUDA graph: replay() runs the same
    library kernels with no host work between the launches.  The plan reads
    its inputs from the device tensors it holds (new data is copied into
    them) and its run() neither synchronises nor allocates outside torch's
    caching allocator, so the captured step is the eager step.  The outputs
    are the tensors of the captured run, rewritten by every replay."""

    def __init__(self, plan, warmup: int = 3):
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):  # workspaces and output pools settle before capture
            for _ in range(warmup):
                plan.run()
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        self.plan = plan
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.out = plan.run()

    def run(self):
        self.graph.replay()
        return self.out


class ShippingPriority:
    """groupjoin=True (the default): one group-join call (dimension filter,
    fact filter, join and GROUP BY key in one pass over the fact rows, groups
    read out in key order) and top-10.  groupjoin=False: the separate path,
    hash build -> probe with gathers -> group-by (`groupby_strategy`) ->
    top-10."""

    def __init__(self, fact: dict, dim: dict, dim_selectivity: float = 0.2, groupby_strategy: str = "auto",
                 groupjoin: bool = True):
        self.f = fact  # key, price, disc, date
        self.d = dim   # key, segment
        self.groupjoin = groupjoin
        # the join key is bounded by the dimension's key range 1..n_dim: AUTO
        # takes the partition strategy ("sort" keeps the general sort)
        self.groupby_strategy = groupby_strategy
        dev = fact["key"].device
        self.n_fact = fact["key"].numel()
        self.n_dim = dim["key"].numel()
        # hash table sized from the expected build count (segment = 2 of U[0,4])
        self.nslots = ops.join_default_slots(int(self.n_dim * dim_selectivity * 1.05))
        self.table = torch.empty(self.nslots, dtype=torch.int64, device=dev)
        # probe output capacity: every fact row (host-side upper bound)
        self.cap = self.n_fact
        self.status = ops.new_status(dev)
        # group-join: dimension keys bounded by 1..n_dim (the key metadata)
        self.gj = ops.GroupJoin(self.n_dim, 1, self.n_dim, [("sum_mul_kminus", 2, 3, 100)], topk=10, topk_agg=0,
                                device=dev) if groupjoin else None

    def run(self):
        if self.groupjoin:
            return self.run_groupjoin()
        st = self.status
        ops.join_build([self.d["key"], self.d["segment"]], 0, preds=[(1, "==", 2)], nslots=self.nslots,
                       table=self.table, status=st)
        pr = ops.join_probe(self.table, [self.f["key"], self.f["date"], self.f["price"], self.f["disc"]], 0,
                            preds=[(1, ">", 1200)], gather=[0, 2, 3], capacity=self.cap, rowids=False,
                            payload=False, status=st)
        self.last_probe = pr
        key_c, price_c, disc_c = pr["gathered"]
        gb = ops.groupby_agg([ops.Col(key_c, 1, self.n_dim), price_c, disc_c], [0],
                             [("sum_mul_kminus", 1, 2, 100)], n=self.cap, nsel=pr["count"],
                             strategy=self.groupby_strategy,
                             capacity=self.cap, status=st)
        ov, okk, dk = ops.topk(gb["aggs"][0], gb["keys"][0], 10, d_n=gb["ngroups"], status=st)
        return {"top_vals": ov, "top_keys": okk, "k": dk, "ngroups": gb["ngroups"], "nmatch": pr["count"],
                "groups": gb, "status": st}

    # the three steps of the group-join plan (timed one by one by the benchmark)
    def gj_build(self):
        self.gj.build([self.d["key"], self.d["segment"]], 0, preds=[(1, "==", 2)], status=self.status)

    def gj_probe(self):
        self.gj.probe([self.f["key"], self.f["date"], self.f["price"], self.f["disc"]], 0, preds=[(1, ">", 1200)],
                      status=self.status)

    def gj_finish(self):
        gb = self.gj.finish(status=self.status)
        return {"top_vals": gb["top_vals"], "top_keys": gb["top_keys"], "k": gb["k"], "ngroups": gb["ngroups"],
                "nmatch": gb["nmatch"], "groups": gb, "status": self.status}

    def run_groupjoin(self):
        self.gj_build()
        self.gj_probe()
        return self.gj_finish()


class JoinChain:
    """fused=True: the last join and the GROUP BY category run as one
    probe + aggregate call.  fused=False: the last probe writes (category,
    payload) per matched probe row and a separate group-by (groupby_strategy,
    e.g. "sort" for the onesweep radix-sort path) aggregates them."""

    def __init__(self, d: dict, n_category: int = 100000, fused: bool = True, groupby_strategy: str = "auto"):
        self.d = d  # third_pk, third_cat, build_pk, build_fk2, probe_fk, probe_payload
        self.fused = fused
        self.groupby_strategy = groupby_strategy
        dev = d["probe_fk"].device
        self.n_third = d["third_pk"].numel()
        self.n_build = d["build_pk"].numel()
        self.n_probe = d["probe_fk"].numel()
        self.n_category = n_category
        self.t1 = torch.empty(ops.join_default_slots(self.n_third), dtype=torch.int64, device=dev)
        self.t2 = torch.empty(ops.join_default_slots(self.n_build), dtype=torch.int64, device=dev)
        self.status = ops.new_status(dev)

    def run(self):
        st = self.status
        d = self.d
        ops.join_build([d["third_pk"], d["third_cat"]], 0, payload_col=1, table=self.t1, nslots=self.t1.numel(),
                       status=st)
        p1 = ops.join_probe(self.t1, [d["build_fk2"], d["build_pk"]], 0, gather=[1], capacity=self.n_build,
                            rowids=False, status=st)
        ops.join_build([p1["gathered"][0], p1["payload"]], 0, payload_col=1, n=self.n_build, d_n=p1["count"],
                       table=self.t2, nslots=self.t2.numel(), status=st)
        if self.fused:
            out = ops.join_probe_agg(self.t2, [d["probe_fk"], d["probe_payload"]], 0, 0, self.n_category - 1,
                                     [("sum", 1), ("count",)], status=st)
        else:
            p2 = ops.join_probe(self.t2, [d["probe_fk"], d["probe_payload"]], 0, gather=[1], capacity=self.n_probe,
                                rowids=False, status=st)
            gb = ops.groupby_agg([ops.Col(p2["payload"], 0, self.n_category - 1), p2["gathered"][0]], [0],
                                 [("sum", 1), ("count",)], n=self.n_probe, nsel=p2["count"],
                                 strategy=self.groupby_strategy, capacity=self.n_category, status=st)
            out = {"keys": gb["keys"][0], "aggs": gb["aggs"], "ngroups": gb["ngroups"], "status": st,
                   "probe_matches": p2["count"]}
        out["build_matches"] = p1["count"]
        return out


class SoftQuery:
    def __init__(self, d: dict, n_groups: int = 1024, tau: float = 0.1):
        self.d = d  # x, v, gid
        dev = d["x"].device
        self.G = n_groups
        self.tau = tau
        self.theta = torch.zeros(n_groups, dtype=torch.float32, device=dev)
        self.gS = torch.ones(n_groups, dtype=torch.float32, device=dev)
        self.gC = torch.ones(n_groups, dtype=torch.float32, device=dev)

    def run(self):
        d = self.d
        S, C = ops.soft_agg_fwd(d["x"], d["v"], d["gid"], self.theta, self.tau)
        gth, _, _ = ops.soft_agg_bwd(d["x"], d["v"], d["gid"], self.theta, self.tau, self.gS, self.gC)
        return S, C, gth
