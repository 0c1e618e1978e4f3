"""Writes tests/golden/plans_expected.json: the oracle's results for the
benchmark plans at sizes too large to recompute inside a GPU test run.

Only ``gen`` (seeded inputs) and ``oracle`` are used; nothing here touches
the CUDA path.  For each case the file holds the scalar results (match and
group counts, the top-10), SHA-256 digests of the whole key and aggregate
columns (bit-exact comparison of every element), and a sample of groups at
fixed positions so that a mismatch shows where it starts.

Cases (the plans of the benchmark, Sec. 2 relational operators):
  shipping_quarter / shipping_full
      dimension WHERE segment = 2, fact WHERE date > 1200, inner join on key,
      GROUP BY key SUM(price * (100 - disc)), top-10 by sum desc, key asc;
      15M x 3.75M and 60M x 15M rows.
  chain_quarter / chain_full
      third (pk -> category) <- build.fk2; build (pk -> category) <- probe.fk;
      GROUP BY category SUM(payload), COUNT(*); 25M / 2.5M / 250k and
      100M / 10M / 1M rows.
  pricing_60M
      WHERE date <= 2460 GROUP BY flag, status: SUM qty, SUM price,
      SUM price*(100-disc), COUNT, AVG qty over 60M rows.

Usage: python tests/golden/make_plan_expected.py [case ...]
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import gen  # noqa: E402
from oracle import relational as R  # noqa: E402

OUT = os.path.join(HERE, "plans_expected.json")
SAMPLE = 25


def digest(a, dtype) -> str:
    return hashlib.sha256(np.ascontiguousarray(a, dtype=dtype).tobytes()).hexdigest()


def sample_idx(n: int):
    if n == 0:
        return []
    return sorted(set(np.linspace(0, n - 1, SAMPLE).astype(np.int64).tolist()))


def shipping(nf: int, nd: int) -> dict:
    seed = gen.BASE_SEED + 1
    fact = gen.fact_table(nf, nd, seed, cols=("key", "price", "disc", "date"))
    dim = gen.dim_table(nd, seed, cols=("key", "segment"))
    bsel = R.filter([(dim["segment"], "==", 2)], nd)
    psel = R.filter([(fact["date"], ">", 1200)], nf)
    # the dimension keys are unique, so a probe row matches at most once
    prow, _, dup = R.join(dim["key"], fact["key"], bsel=bsel, psel=psel, cap=len(psel))
    assert not dup
    keys, aggs = R.groupby([fact["key"]], [("sum_mul_kminus", fact["price"], fact["disc"], 100)], nf, sel=prow)
    tv, tk = R.topk(aggs[:, 0], keys[:, 0], 10)
    g = len(keys)
    idx = sample_idx(g)
    return {"fact_rows": nf, "dim_rows": nd, "seed": seed, "nmatch": int(len(prow)), "ngroups": int(g),
            "keys_sha256": digest(keys[:, 0], np.int32), "sums_sha256": digest(aggs[:, 0], np.int64),
            "sample_idx": idx, "sample_keys": [int(keys[i, 0]) for i in idx],
            "sample_sums": [int(aggs[i, 0]) for i in idx],
            "top_vals": [int(v) for v in tv], "top_keys": [int(k) for k in tk]}


def chain(n_probe: int, n_build: int, n_third: int) -> dict:
    seed = gen.BASE_SEED + 2
    d = gen.chain_tables(n_probe, n_build, n_third, seed)
    # build rows find their category through the third table
    b_rows, t_rows, dup1 = R.join(d["third_pk"], d["build_fk2"], cap=n_build)
    assert not dup1
    cat_of = d["third_cat"][t_rows]
    # probe rows find their build row (and so its category)
    pk = d["build_pk"][b_rows]
    p_rows, ib, dup2 = R.join(pk, d["probe_fk"].astype(np.int32), cap=n_probe)
    assert not dup2
    cat = np.ascontiguousarray(cat_of[ib], dtype=np.int32)
    pay = np.ascontiguousarray(d["probe_payload"][p_rows])
    keys, aggs = R.groupby([cat], [("sum", pay, None, None), ("count", None, None, None)], len(cat))
    g = len(keys)
    idx = sample_idx(g)
    return {"probe_rows": n_probe, "build_rows": n_build, "third_rows": n_third, "seed": seed,
            "build_matches": int(len(b_rows)), "probe_matches": int(len(p_rows)), "ngroups": int(g),
            "keys_sha256": digest(keys[:, 0], np.int32), "sums_sha256": digest(aggs[:, 0], np.int64),
            "counts_sha256": digest(aggs[:, 1], np.int64),
            "sample_idx": idx, "sample_keys": [int(keys[i, 0]) for i in idx],
            "sample_sums": [int(aggs[i, 0]) for i in idx], "sample_counts": [int(aggs[i, 1]) for i in idx]}


def pricing(n: int) -> dict:
    seed = gen.BASE_SEED + 1
    t = gen.fact_table(n, 15_000_000, seed, cols=("flag", "status", "qty", "price", "disc", "date"))
    sel = R.filter([(t["date"], "<=", 2460)], n)
    keys, aggs = R.groupby([t["flag"], t["status"]],
                           [("sum", t["qty"], None, None), ("sum", t["price"], None, None),
                            ("sum_mul_kminus", t["price"], t["disc"], 100), ("count", None, None, None),
                            ("avg", t["qty"], None, None)], n, sel=sel)
    return {"rows": n, "seed": seed, "selected": int(len(sel)), "keys": keys.tolist(), "aggs": aggs.tolist()}


CASES = {
    "shipping_quarter": lambda: shipping(15_000_000, 3_750_000),
    "shipping_full": lambda: shipping(60_000_000, 15_000_000),
    "chain_quarter": lambda: chain(25_000_000, 2_500_000, 250_000),
    "chain_full": lambda: chain(100_000_000, 10_000_000, 1_000_000),
    "pricing_60M": lambda: pricing(60_000_000),
}


def main(names):
    res = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            res = json.load(f)
    res["about"] = ("Oracle results (oracle/ only, inputs from gen) for the benchmark plans; written by "
                    "tests/golden/make_plan_expected.py.")
    for name in names or list(CASES):
        t0 = time.time()
        res[name] = CASES[name]()
        print("%s: %.1f s" % (name, time.time() - t0), flush=True)
        with open(OUT, "w") as f:
            json.dump(res, f, indent=1)


if __name__ == "__main__":
    main(sys.argv[1:])
