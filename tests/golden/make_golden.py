"""Writes the golden fixtures of this directory from the oracle alone (never
from the CUDA path): the star query of the workloads (filter, PK-FK join
(Section 3.2), group-by with exact 128-bit decimal sums and AVG (Section 4))
on small seeded inputs, and the modular dataset whose per-group values also
follow from arithmetic series.  Run from the repository root:

    python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle                                   # noqa: E402
from datagen import workloads as W              # noqa: E402

CASES = {
    "star_lowcard_20k.txt": lambda: W.config1(n_fact=20_000, n_dim=1_000),
    "modular_11550.txt": lambda: W.modular(11_550, 200),
}


def render(wl) -> str:
    r = oracle.run(wl)
    aggs = wl.query["aggs"]
    lines = [f"# {wl.name}: {wl.n_fact} fact rows, {wl.n_dim} dimension rows; query {wl.query}",
             "# key count then per aggregate its exact sum (decimal), and the AVG as a hex double where there is one"]
    for g in range(r.n_groups):
        cols = [str(int(r.keys[g])), str(int(r.counts[g]))]
        for a, ag in enumerate(aggs):
            cols.append(str(r.sum_int(g, a)))
            if ag[0] == "avg":
                cols.append(float(r.avgs[g, a]).hex())
        lines.append(" ".join(cols))
    return "\n".join(lines) + "\n"


def main():
    for name, make in CASES.items():
        with open(os.path.join(HERE, name), "w") as f:
            f.write(render(make()))
        print("wrote", name)


if __name__ == "__main__":
    main()
