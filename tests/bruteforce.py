"""Brute-force evaluation for tiny inputs: a nested-loop join and a linear
scan over a list of groups, in Python integers.  Used to pin the oracle."""
from __future__ import annotations


def _val(arr, i):
    return int(arr[i])


def evaluate(fact: dict, dim: dict | None, query: dict, extra_dims: list | None = None):
    """Returns a list of (key, count, [sum per agg], [avg per agg or None]),
    sorted by key; raises ValueError('dup_key' | 'range').  A star join lists
    further joins in query["extra_joins"] over the tables extra_dims."""
    n_fact = len(next(iter(fact.values()))) if fact else 0
    # every joined dimension: (table, join, predicate), the first one first
    sides = []
    if query.get("join") is not None:
        sides.append((dim, query["join"], query.get("dim_filter")))
        for j, xj in enumerate(query.get("extra_joins") or []):
            sides.append((extra_dims[j], xj, xj.get("dim_filter")))
    names = {"dim": 0, "dim1": 1, "dim2": 2, "dim3": 3}
    live, pks = [], []
    for tab, join, dflt in sides:
        n_dim = len(next(iter(tab.values()))) if tab else 0
        # dimension rows the dimension predicate admits (all when there is none)
        lv = [dflt is None or dflt["lo"] <= _val(tab[dflt["col"]], d) <= dflt["hi"] for d in range(n_dim)]
        pk = [int(x) for x in tab[join["dim_col"]]] if tab else []
        for a in range(n_dim):
            for b in range(a + 1, n_dim):
                if lv[a] and lv[b] and pk[a] == pk[b] and not join.get("many"):
                    raise ValueError("dup_key")
        live.append(lv)
        pks.append(pk)
    groups = []  # list of [key, count, sums]
    aggs = query["aggs"]
    flt = query.get("filter")
    for i in range(n_fact):
        if flt is not None:
            v = _val(fact[flt["col"]], i)
            if not (flt["lo"] <= v <= flt["hi"]):
                continue
        combos = [[]]     # every combination of partner rows, one per dimension
        for k, (tab, join, _) in enumerate(sides):
            fk = _val(fact[join["fact_col"]], i)
            rows = [d for d in range(len(pks[k])) if live[k][d] and pks[k][d] == fk]
            combos = [c + [d] for c in combos for d in rows]
        for ds in combos:
            key = 0
            for side, col, bits in query["group"]:
                v = _val(fact[col], i) if side == "fact" else _val(sides[names[side]][0][col], ds[names[side]])
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
