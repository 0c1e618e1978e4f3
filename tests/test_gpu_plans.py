"""Whole benchmark plans on the GPU against the oracle, bit-exact.

Small plans are compared with the oracle computed in the test.  The
benchmark-size plans (the shipping-priority plan at 1/4 and full size, the
three-table join chain at 1/4 and full size, the 60M-row pricing summary)
are compared with the oracle's results stored in tests/golden/
plans_expected.json by tests/golden/make_plan_expected.py (oracle/ and gen
only): counts and top-10 directly, every group key and aggregate through a
SHA-256 digest of the whole column, plus a fixed sample of groups.
"""
import hashlib
import json
import os

import numpy as np
import pytest
import torch

import gen
from oracle import relational as R
from paper_2211_02753_b300 import ops, plans

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "plans_expected.json")


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def np_(t, n=None):
    a = t.cpu().numpy()
    return a if n is None else a[:n]


def sha(a, dtype):
    return hashlib.sha256(np.ascontiguousarray(a, dtype=dtype).tobytes()).hexdigest()


def gold(name):
    with open(GOLD) as f:
        d = json.load(f)
    if name not in d:
        pytest.fail("no stored oracle result for %s" % name)
    return d[name]


def _shipping_inputs(nf, nd, seed):
    fact = {k: cu(v) for k, v in gen.fact_table(nf, nd, seed, cols=("key", "price", "disc", "date")).items()}
    dim = {k: cu(v) for k, v in gen.dim_table(nd, seed, cols=("key", "segment")).items()}
    return fact, dim


def _shipping_result(o):
    g = int(o["ngroups"].item())
    return {"nmatch": int(o["nmatch"].item()), "ngroups": g, "keys": np_(o["groups"]["keys"][0], g),
            "sums": np_(o["groups"]["aggs"][0], g), "k": int(o["k"].item()),
            "top_vals": np_(o["top_vals"]), "top_keys": np_(o["top_keys"])}


STRATEGIES = ["groupjoin", "auto", "sort"]


def _plan(fact, dim, strategy):
    if strategy == "groupjoin":
        return plans.ShippingPriority(fact, dim, groupjoin=True)
    return plans.ShippingPriority(fact, dim, groupjoin=False, groupby_strategy=strategy)


@pytest.mark.parametrize("strategy", STRATEGIES)
def test_shipping_plan_small_matches_oracle(strategy):
    nf, nd, seed = 1_000_003, 250_001, 31
    fact_h = gen.fact_table(nf, nd, seed, cols=("key", "price", "disc", "date"))
    dim_h = gen.dim_table(nd, seed, cols=("key", "segment"))
    fact, dim = {k: cu(v) for k, v in fact_h.items()}, {k: cu(v) for k, v in dim_h.items()}
    p = _plan(fact, dim, strategy)
    got = _shipping_result(p.run())
    ops.check(p.status)
    bsel = R.filter([(dim_h["segment"], "==", 2)], nd)
    psel = R.filter([(fact_h["date"], ">", 1200)], nf)
    prow, _, dup = R.join(dim_h["key"], fact_h["key"], bsel=bsel, psel=psel)
    assert not dup
    keys, aggs = R.groupby([fact_h["key"]], [("sum_mul_kminus", fact_h["price"], fact_h["disc"], 100)], nf,
                           sel=prow)
    tv, tk = R.topk(aggs[:, 0], keys[:, 0], 10)
    assert got["nmatch"] == len(prow)
    assert got["ngroups"] == len(keys)
    assert np.array_equal(got["keys"], keys[:, 0])
    assert np.array_equal(got["sums"], aggs[:, 0])
    assert got["k"] == 10
    assert np.array_equal(got["top_vals"], tv) and np.array_equal(got["top_keys"], tk)


def _check_shipping_gold(got, e):
    assert got["nmatch"] == e["nmatch"]
    assert got["ngroups"] == e["ngroups"]
    idx = e["sample_idx"]
    assert got["keys"][idx].tolist() == e["sample_keys"]
    assert got["sums"][idx].tolist() == e["sample_sums"]
    assert sha(got["keys"], np.int32) == e["keys_sha256"]
    assert sha(got["sums"], np.int64) == e["sums_sha256"]
    assert got["top_vals"].tolist() == e["top_vals"]
    assert got["top_keys"].tolist() == e["top_keys"]


@pytest.mark.parametrize("case", ["shipping_quarter", "shipping_full"])
def test_shipping_plan_benchmark_size_matches_oracle(case):
    """The headline plan at 1/4 and at full size (60M x 15M rows: 6.36M
    matches, 2.64M groups), every strategy, against the stored oracle
    result; the full size also through the CUDA-graph replay the benchmark
    times."""
    e = gold(case)
    fact, dim = _shipping_inputs(e["fact_rows"], e["dim_rows"], e["seed"])
    for strategy in STRATEGIES:
        p = _plan(fact, dim, strategy)
        _check_shipping_gold(_shipping_result(p.run()), e)
        ops.check(p.status, case + " " + strategy)
        if case == "shipping_full" and strategy == "groupjoin":
            step = plans.Graphed(p)
            _check_shipping_gold(_shipping_result(step.run()), e)
            ops.check(p.status, case + " graph")
        del p
        torch.cuda.empty_cache()


@pytest.mark.parametrize("case", ["chain_quarter", "chain_full"])
def test_join_chain_plan_matches_oracle(case):
    """The three-table chain (Zipf(1.0) probes into the build table, which
    reaches the third table through Zipf(0.5) keys; a build fed by the
    count of the first probe's output) against the stored oracle result."""
    e = gold(case)
    d = gen.chain_tables(e["probe_rows"], e["build_rows"], e["third_rows"], e["seed"])
    dd = {k: cu(v.astype(np.int32) if k == "probe_fk" else v) for k, v in d.items()}
    del d
    # fused probe + group-by, and the separate probe -> group-by on the
    # onesweep sort path and on the small-domain path
    for fused, strategy in ((True, "auto"), (False, "sort"), (False, "small_domain")):
        jc = plans.JoinChain(dd, fused=fused, groupby_strategy=strategy)
        out = jc.run()
        ops.check(jc.status, "%s fused=%s %s" % (case, fused, strategy))
        assert int(out["build_matches"].item()) == e["build_matches"]
        if not fused:
            assert int(out["probe_matches"].item()) == e["probe_matches"]
        g = int(out["ngroups"].item())
        assert g == e["ngroups"]
        keys, sums, cnts = np_(out["keys"], g), np_(out["aggs"][0], g), np_(out["aggs"][1], g)
        idx = e["sample_idx"]
        assert keys[idx].tolist() == e["sample_keys"]
        assert sums[idx].tolist() == e["sample_sums"]
        assert cnts[idx].tolist() == e["sample_counts"]
        assert int(cnts.sum()) == e["probe_matches"]
        assert sha(keys, np.int32) == e["keys_sha256"]
        assert sha(sums, np.int64) == e["sums_sha256"]
        assert sha(cnts, np.int64) == e["counts_sha256"]
        del jc, out
        torch.cuda.empty_cache()


def test_pricing_summary_60M_both_strategies_match_oracle():
    """WHERE date <= 2460 GROUP BY flag, status over 60M rows, on the
    small-domain path and on the onesweep sort path, against the oracle."""
    e = gold("pricing_60M")
    t = gen.fact_table(e["rows"], 15_000_000, e["seed"], cols=("flag", "status", "qty", "price", "disc", "date"))
    td = {k: cu(v) for k, v in t.items()}
    del t
    for strategy in ("small_domain", "sort"):
        p = plans.PricingSummary(td, strategy)
        out = p.run()
        ops.check(out["status"], strategy)
        g = int(out["ngroups"].item())
        assert g == len(e["keys"])
        keys = np.stack([np_(k, g).astype(np.int64) for k in out["keys"]], 1)
        aggs = np.stack([np_(a, g) for a in out["aggs"]], 1)
        assert keys.tolist() == e["keys"]
        assert aggs.tolist() == e["aggs"]


@pytest.mark.parametrize("n,bits", [(6_400_000, 24), (12_800_001, 64)])
def test_sort_pairs_large_matches_oracle(n, bits):
    """The onesweep radix sort across thousands of tiles and their look-back
    chain, at the sizes of the headline group-by input and beyond."""
    r = np.random.default_rng(n + bits)
    if bits < 64:
        keys = r.integers(0, 1 << bits, n, dtype=np.uint64)
    else:
        keys = r.integers(0, 2**63, n).astype(np.uint64) * 2 + r.integers(0, 2, n).astype(np.uint64)
    keys[n // 5: n // 5 + n // 4] = keys[7]  # a long run of equal keys (stability across tiles)
    vals = np.arange(n, dtype=np.uint32)
    ko, vo, st = ops.sort_pairs(cu(keys.view(np.int64)), cu(vals.view(np.int32)), key_bits=bits)
    ops.check(st)
    ek, ev = R.sort_pairs(keys, vals)
    assert np.array_equal(np_(ko).view(np.uint64), ek)
    assert np.array_equal(np_(vo).view(np.uint32), ev)
