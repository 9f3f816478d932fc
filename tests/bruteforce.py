"""Brute-force evaluation for tiny inputs: a nested-loop join and a linear
scan over a list of groups, in Python integers.  Used to pin the oracle."""
from __future__ import annotations


def _val(arr, i):
    return int(arr[i])


def evaluate(fact: dict, dim: dict | None, query: dict):
    """Returns a list of (key, count, [sum per agg], [avg per agg or None]),
    sorted by key; raises ValueError('dup_key' | 'range')."""
    n_fact = len(next(iter(fact.values()))) if fact else 0
    n_dim = len(next(iter(dim.values()))) if dim else 0
    join = query.get("join")
    dflt = query.get("dim_filter")
    # dimension rows the dimension predicate admits (all when there is none)
    live = [dflt is None or dflt["lo"] <= _val(dim[dflt["col"]], d) <= dflt["hi"] for d in range(n_dim)]
    if join is not None:
        pk = [int(x) for x in dim[join["dim_col"]]] if dim else []
        for a in range(n_dim):
            for b in range(a + 1, n_dim):
                if live[a] and live[b] and pk[a] == pk[b]:
                    raise ValueError("dup_key")
    groups = []  # list of [key, count, sums]
    aggs = query["aggs"]
    flt = query.get("filter")
    for i in range(n_fact):
        if flt is not None:
            v = _val(fact[flt["col"]], i)
            if not (flt["lo"] <= v <= flt["hi"]):
                continue
        partners = [None]
        if join is not None:
            fk = _val(fact[join["fact_col"]], i)
            partners = [d for d in range(n_dim) if live[d] and pk[d] == fk]
        for d in partners:
            key = 0
            for side, col, bits in query["group"]:
                v = _val(fact[col], i) if side == "fact" else _val(dim[col], d)
                if bits < 64:
                    if not (0 <= v < (1 << bits)):
                        raise ValueError("range")
                    key = (key << bits) | v
                else:
                    key = v & ((1 << 64) - 1)
            terms = []
            for ag in aggs:
                if ag[0] in ("sum", "avg"):
                    terms.append(_val(fact[ag[1]], i))
                elif ag[0] == "sum_mul_sub":
                    terms.append(_val(fact[ag[1]], i) * (ag[2] - _val(fact[ag[3]], i)))
                else:
                    terms.append(1)
            for g in groups:          # linear scan over the groups seen so far
                if g[0] == key:
                    g[1] += 1
                    for k, t in enumerate(terms):
                        g[2][k] += t
                    break
            else:
                groups.append([key, 1, list(terms)])
    out = []
    for key, count, sums in sorted(groups, key=lambda g: g[0]):
        # AVG: the exact sum and the count each rounded to double, then one
        # IEEE division
        avgs = [(float(s) / float(count) if ag[0] == "avg" else None) for s, ag in zip(sums, aggs)]
        out.append((key, count, sums, avgs))
    return out
