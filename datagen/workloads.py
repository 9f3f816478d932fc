"""Synthetic star-schema workloads: seeded tables plus the query each one runs.

The shapes stand in for the paper's TPC-H runs (Section 4: lineitem-like fact
rows joined to an orders/part-like dimension, a 2,557-day date domain, 3- and
2-valued flags, decimal(11,2) money held as scaled integers).  No TPC item is
reproduced.  Only data and query *descriptions* live here; nothing evaluates a
query.

Query description (a plain dict, translated by each side into its own plan):
  filter : {"col", "lo", "hi"}  inclusive bounds on a fact column, or None
  join   : {"fact_col", "dim_col"}  PK-FK inner equi-join, or None
  group  : [(side, col, bits), ...]  packed first-field-highest into <= 64 bits
  aggs   : ("sum", col) | ("sum_mul_sub", a, K, b) | ("count",) | ("avg", col)

Scaled decimals: qty = units*100, price = cents, disc = percent (0..10), so
SUM(price*(100-disc)) is at scale 10^4.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import (IOTA, MODULAR, PERM, PERM_DIV, RAW64, fill, gather, index, loguniform, lognormal,
               raw_at, uniform, zipf_cdf)

I64_MIN = -(1 << 63)
I64_MAX = (1 << 63) - 1
N_DAYS = 2557          # 7 years of day indices 0..2556
CUTOFF_98 = 2504       # date <= 2504 keeps 2505/2557 = 97.97% of uniform dates
RANGE_1PCT = 25        # [lo, lo + 25] keeps 26/2557 = 1.02%

SEEDS = {1: 0x7E5E0001, 2: 0x7E5E0002, 3: 0x7E5E0003, 4: 0x7E5E0004, 5: 0x7E5E0005}

# stream ids: table * 64 + column
_FACT, _DIM, _META, _XDIM = 0, 1, 2, 3
S_FK, S_DATE, S_QTY, S_PRICE, S_DISC, S_FLAG, S_STATUS, S_OKEY, S_FKX = range(9)
S_PK, S_ATTR, S_BAND = 0, 1, 2


def _s(table, col, sub=0):
    return table * 64 + col + sub * 4096


@dataclass
class Workload:
    name: str
    fact: dict                      # name -> np.ndarray (all the same length)
    dim: dict | None                # name -> np.ndarray, or None
    query: dict
    meta: dict = field(default_factory=dict)

    @property
    def n_fact(self) -> int:
        return len(next(iter(self.fact.values())))

    @property
    def n_dim(self) -> int:
        return 0 if self.dim is None else len(next(iter(self.dim.values())))


def q_lowcard(cutoff=CUTOFF_98, attr_bits=5):
    """Filter date <= cutoff, join fk = pk, group by (flag, status, attr),
    SUM(qty), SUM(price*(100-disc)), COUNT(*), AVG(disc)."""
    return dict(
        filter=dict(col="date", lo=I64_MIN, hi=int(cutoff)),
        join=dict(fact_col="fk", dim_col="pk"),
        group=[("fact", "flag", 2), ("fact", "status", 1), ("dim", "attr", attr_bits)],
        aggs=[("sum", "qty"), ("sum_mul_sub", "price", 100, "disc"), ("count",), ("avg", "disc")],
    )


def q_highcard(lo, hi):
    """Filter lo <= date <= hi, join fk = pk, group by orderkey, SUM(price*(100-disc))."""
    return dict(
        filter=dict(col="date", lo=int(lo), hi=int(hi)),
        join=dict(fact_col="fk", dim_col="pk"),
        group=[("fact", "okey", 64)],
        aggs=[("sum_mul_sub", "price", 100, "disc"), ("count",)],
    )


def _measures(seed, n, row0=0):
    return dict(
        date=uniform(seed, _s(_FACT, S_DATE), np.int32, n, 0, N_DAYS - 1, row0=row0),
        qty=uniform(seed, _s(_FACT, S_QTY), np.int64, n, 1, 50, mult=100, row0=row0),
        price=uniform(seed, _s(_FACT, S_PRICE), np.int64, n, 90_000, 10_500_000, row0=row0),
        disc=uniform(seed, _s(_FACT, S_DISC), np.int64, n, 0, 10, row0=row0),
        flag=uniform(seed, _s(_FACT, S_FLAG), np.uint8, n, 0, 2, row0=row0),
        status=uniform(seed, _s(_FACT, S_STATUS), np.uint8, n, 0, 1, row0=row0),
    )


def config1(n_fact=1_000_000, n_dim=10_000, seed=SEEDS[1], cutoff=CUTOFF_98) -> Workload:
    """Device-resident single batch: 1M fact rows, 10k-row dimension with pk
    0..n_dim-1, fk uniform over the dimension keys, attr in 25 values."""
    dim = dict(
        pk=fill(seed, _s(_DIM, S_PK), IOTA, np.int32, n_dim),
        attr=uniform(seed, _s(_DIM, S_ATTR), np.int32, n_dim, 0, 24),
    )
    fk = gather(dim["pk"], index(seed, _s(_FACT, S_FK), n_dim, n_fact))
    fact = dict(fk=fk, **_measures(seed, n_fact))
    return Workload("star-1M-lowcard", fact, dim, q_lowcard(cutoff))


def config2_tables(n_fact=60_000_000, n_dim=2_000_000, n_okey=None, seed=SEEDS[2], zipf_s=0.8,
                   sparse_keys=False):
    """60M fact rows (+ int64 orderkey, 4 adjacent rows per key, keys a seeded
    permutation), 2M-row dimension with unique scrambled int32 pk, fk Zipf(s)
    over the dimension rows with the hot rows scattered.  sparse_keys: the
    dimension keys are unique sparse int64 values (raw SplitMix64 outputs) and
    fk is int64, so the join needs a hashed table."""
    if n_okey is None:
        n_okey = max(1, n_fact // 4)
    dim = dict(
        pk=fill(seed, _s(_DIM, S_PK), RAW64, np.int64, n_dim) if sparse_keys else
        fill(seed, _s(_DIM, S_PK), PERM, np.int32, n_dim, b=n_dim),
        attr=uniform(seed, _s(_DIM, S_ATTR), np.int32, n_dim, 0, 24),
    )
    cdf = zipf_cdf(zipf_s, n_dim)
    fk = gather(dim["pk"], index(seed, _s(_FACT, S_FK), n_dim, n_fact, cdf=cdf))
    fact = dict(fk=fk, **_measures(seed, n_fact))
    fact["okey"] = fill(seed, _s(_FACT, S_OKEY), PERM_DIV, np.int64, n_fact, a=2, b=n_okey)
    return fact, dim


def config2_range_lo(seed=SEEDS[2]) -> int:
    return int(uniform(seed, _s(_META, 0), np.int64, 1, 0, N_DAYS - 1 - RANGE_1PCT)[0])


def config2(which="a", **kw) -> Workload:
    """which: 'a' low-cardinality query, 'b' 1%-selective high-cardinality
    query on orderkey, 'b2' the same high-cardinality query at ~98%."""
    seed = kw.get("seed", SEEDS[2])
    fact, dim = config2_tables(**kw)
    if which == "a":
        q = q_lowcard()
    elif which == "b":
        lo = config2_range_lo(seed)
        q = q_highcard(lo, lo + RANGE_1PCT)
    elif which == "b2":
        q = q_highcard(0, CUTOFF_98)
    else:
        raise ValueError(which)
    return Workload(f"star-{len(fact['fk'])}-{which}", fact, dim, q)


def config3_dim(n_dim=150_000_000, seed=SEEDS[3], row0=0, n=None):
    """Build side: unique sparse int64 pk (raw SplitMix64 outputs, distinct per
    row) and int32 attr in 25 values."""
    n = n_dim - row0 if n is None else n
    return dict(
        pk=fill(seed, _s(_DIM, S_PK), RAW64, np.int64, n, row0=row0),
        attr=uniform(seed, _s(_DIM, S_ATTR), np.int32, n, 0, 24, row0=row0),
    )


def config3_fact(row0, n, n_dim=150_000_000, seed=SEEDS[3]):
    """Rows row0..row0+n-1 of the out-of-core fact table: fk int64 uniform over
    the build rows' keys, plus the config-1 measure columns."""
    idx = index(seed, _s(_FACT, S_FK), n_dim, n, row0=row0)
    fk = raw_at(seed, _s(_DIM, S_PK), idx)   # pk of build row j, regenerated
    return dict(fk=fk, **_measures(seed, n, row0=row0))


def config3(n_fact=600_000_000, n_dim=150_000_000, seed=SEEDS[3]) -> Workload:
    dim = config3_dim(n_dim, seed)
    idx = index(seed, _s(_FACT, S_FK), n_dim, n_fact)
    fact = dict(fk=gather(dim["pk"], idx), **_measures(seed, n_fact))
    return Workload(f"star-{n_fact}-outofcore", fact, dim, q_lowcard())


def star_dim(n_dim, seed, j=0):
    """Further dimension j of a star join: unique sparse int64 keys (raw
    SplitMix64 outputs, distinct per row), attr in 25 values, band in 4."""
    return dict(
        pk=fill(seed, _s(_XDIM, S_PK, j), RAW64, np.int64, n_dim),
        attr=uniform(seed, _s(_XDIM, S_ATTR, j), np.int32, n_dim, 0, 24),
        band=uniform(seed, _s(_XDIM, S_BAND, j), np.uint8, n_dim, 0, 3),
    )


def star_fk(n_fact, n_dim, seed, j=0):
    """The fact foreign key into star_dim(n_dim, seed, j): uniform over its rows."""
    idx = index(seed, _s(_FACT, S_FKX, j), n_dim, n_fact)
    return raw_at(seed, _s(_XDIM, S_PK, j), idx)


def config4_sizes(n_queries=256, seed=SEEDS[4], fact_lo=10_000, fact_hi=50_000_000,
                  dim_lo=1_000, dim_hi=1_000_000):
    """Per-query sizes: fact lognormal(ln 5e5, 1.5) clamped, dims log-uniform,
    cutoffs uniform over the date domain, group cardinality log-uniform [4, 1e5]."""
    return dict(
        fact=lognormal(seed, _s(_META, 1), float(np.log(5e5)), 1.5, fact_lo, fact_hi, n_queries),
        dim=loguniform(seed, _s(_META, 2), dim_lo, dim_hi, n_queries),
        cutoff=uniform(seed, _s(_META, 3), np.int64, n_queries, 0, N_DAYS - 1),
        groups=loguniform(seed, _s(_META, 4), 4, 100_000, n_queries),
    )


def config4_query(q, n_fact, n_dim, cutoff, groups, seed=SEEDS[4], fact_scale=1.0) -> Workload:
    """Query q of the batched mix: its own fact and dimension tables; the group
    key is the dimension attribute with ``groups`` distinct values."""
    n_fact = max(1, int(n_fact * fact_scale))
    qseed = seed + (q + 1) * 0x1000
    dim = dict(
        pk=fill(qseed, _s(_DIM, S_PK), PERM, np.int32, n_dim, b=n_dim),
        attr=uniform(qseed, _s(_DIM, S_ATTR), np.int32, n_dim, 0, int(groups) - 1),
    )
    fk = gather(dim["pk"], index(qseed, _s(_FACT, S_FK), n_dim, n_fact))
    fact = dict(fk=fk, **_measures(qseed, n_fact))
    bits = max(1, int(groups - 1).bit_length())
    query = dict(
        filter=dict(col="date", lo=I64_MIN, hi=int(cutoff)),
        join=dict(fact_col="fk", dim_col="pk"),
        group=[("dim", "attr", bits)],
        aggs=[("sum", "qty"), ("sum_mul_sub", "price", 100, "disc"), ("count",), ("avg", "disc")],
    )
    return Workload(f"batch-q{q}", fact, dim, query, meta=dict(groups=int(groups)))


def modular(n_fact, n_dim, seed=0):
    """Closed-form dataset: every column is a residue of the row index, so each
    group's count and sums are arithmetic-series formulas (see tests)."""
    dim = dict(
        pk=fill(seed, 0, IOTA, np.int32, n_dim),
        attr=fill(seed, 0, MODULAR, np.int32, n_dim, a=0, b=25, mult=1),
    )
    fact = dict(
        fk=fill(seed, 0, MODULAR, np.int32, n_fact, a=0, b=n_dim, mult=1),
        date=fill(seed, 0, MODULAR, np.int32, n_fact, a=0, b=N_DAYS, mult=1),
        qty=fill(seed, 0, MODULAR, np.int64, n_fact, a=0, b=50, mult=100, c=100),
        price=fill(seed, 0, MODULAR, np.int64, n_fact, a=0, b=7, mult=1000, c=90_000),
        disc=fill(seed, 0, MODULAR, np.int64, n_fact, a=0, b=11, mult=1),
        flag=fill(seed, 0, MODULAR, np.uint8, n_fact, a=0, b=3, mult=1),
        status=fill(seed, 0, MODULAR, np.uint8, n_fact, a=0, b=2, mult=1),
    )
    return Workload(f"modular-{n_fact}x{n_dim}", fact, dim, q_lowcard(cutoff=N_DAYS - 1))
