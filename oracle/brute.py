"""Pure-Python brute force for tiny tables (a few hundred rows).

TEST INFRASTRUCTURE ONLY.  Independent restatement of the SQL semantics used
to pin the C oracle: nested loops for joins, a dict for GROUP BY, Python's
sorted() for top-k, exact rational arithmetic for AVG.
"""
from fractions import Fraction

OPS = {
    "<": lambda a, b: a < b, "<=": lambda a, b: a <= b, ">": lambda a, b: a > b,
    ">=": lambda a, b: a >= b, "==": lambda a, b: a == b, "!=": lambda a, b: a != b,
}


def filter(preds, n):
    return [i for i in range(n) if all(OPS[o](int(c[i]), int(v)) for c, o, v in preds)]


def avg_half_away(s, c):
    """Round s/c to the nearest integer, halves away from zero (exact)."""
    q = Fraction(int(s), int(c))
    mag = abs(q)
    r = int(mag + Fraction(1, 2))  # floor(|q| + 1/2)
    return r if q >= 0 else -r


def groupby(keys, aggs, rows):
    groups = {}
    for r in rows:
        groups.setdefault(tuple(int(k[r]) for k in keys), []).append(r)
    out = []
    for key in sorted(groups):
        rs = groups[key]
        vals = []
        for op, a, b, k in aggs:
            if op == "count":
                vals.append(len(rs))
            elif op == "sum":
                vals.append(sum(int(a[r]) for r in rs))
            elif op == "sum_mul_kminus":
                vals.append(sum(int(a[r]) * (int(k) - int(b[r])) for r in rs))
            elif op == "avg":
                vals.append(avg_half_away(sum(int(a[r]) for r in rs), len(rs)))
            elif op == "min":
                vals.append(min(int(a[r]) for r in rs))
            elif op == "max":
                vals.append(max(int(a[r]) for r in rs))
        out.append((key, tuple(vals)))
    return out


def join(bkey, brows, pkey, prows):
    """Nested loop: for each probe row in order, each build row in order."""
    out = []
    for p in prows:
        for b in brows:
            if int(pkey[p]) == int(bkey[b]):
                out.append((p, b))
    return out


def topk(vals, keys, k):
    items = sorted(zip((int(v) for v in vals), (int(x) for x in keys)), key=lambda t: (-t[0], t[1]))
    return items[:k]
