"""Seeded, counter-based synthetic inputs for the Crystal operators and their oracle.

This module holds input generation only: no step of any query operator is computed
here.  Every value is a pure function of (seed, stream, index), so a test can recompute
any single input element on the host without materialising a whole column, and the
device generator in ``datagen/gen.cu`` (same definitions, checked element-for-element
against this file by the tests) can fill multi-GB columns directly in HBM.

Definitions
-----------
* ``mix64`` is the SplitMix64 output function (Steele, Lea & Flood, "Fast splittable
  pseudorandom number generators", OOPSLA 2014): two xor-shift-multiply rounds and a
  final xor-shift with the published constants.
* The 64-bit word of stream ``s`` at index ``i`` is SplitMix64 evaluated at counter
  ``i``: ``mix64(base + (i + 1) * GAMMA)`` with ``GAMMA = 0x9E3779B97F4A7C15`` and
  ``base = mix64(seed ^ mix64(s))`` (all arithmetic mod 2^64).
* Integers uniform in ``[lo, hi]``: ``lo + (((w >> 32) * (hi - lo + 1)) >> 32)``
  (Lemire's multiply-shift range reduction, without rejection; the bias is below
  2^-32 per value and identical on both sides).
* Floats uniform in ``[0, 1)``: ``(w >> 40) * 2^-24`` (exact float32 values).
* Raw 32-bit patterns: ``int32(w >> 32)``.
* Permutations of ``[0, n)``: a 4-round balanced Feistel network on ``[0, 2^k)``
  (``k`` the smallest even number >= max(2, bitlen(n - 1))), round function
  ``mix64(R + key_r) & (2^(k/2) - 1)`` with ``key_r`` the stream's words 0..3, made a
  permutation of ``[0, n)`` by cycle walking (Black & Rogaway, "Ciphers with
  arbitrary finite domains", CT-RSA 2002).  Element ``j`` of the permutation is
  computable on its own, which is how dense shuffled dimension keys are produced.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_U64 = np.uint64

# Stream ids of every synthetic column.  A column is identified by (seed, stream);
# the device generator receives the same numbers.
STREAMS = {
    # fused filter-probe-aggregate, small (fact 2^22, date-like dimension 2556 rows)
    "q1.fk": 101, "q1.a": 102, "q1.b": 103, "q1.c": 104, "q1.dim_key": 110,
    # operator microbenchmarks on 2^29-row columns
    "sel.x": 201, "proj.x1": 202, "proj.x2": 203,
    # hash join: build keys/values, probe foreign keys/payloads
    "join.bkey": 301, "join.bval": 302, "join.fk": 303, "join.pay": 304,
    # radix sort keys
    "sort.key": 401,
    # served star schema: fact columns 501..508, dimension keys/attributes 510..
    "ss.fk_date": 501, "ss.fk_supp": 502, "ss.fk_cust": 503, "ss.fk_part": 504,
    "ss.qty": 505, "ss.disc": 506, "ss.price": 507, "ss.cost": 508,
    "ss.date.key": 510, "ss.date.year": 511, "ss.date.month": 512,
    "ss.supp.key": 520, "ss.supp.region": 521, "ss.supp.nation": 522, "ss.supp.city": 523,
    "ss.cust.key": 530, "ss.cust.region": 531, "ss.cust.nation": 532, "ss.cust.city": 533,
    "ss.part.key": 540, "ss.part.mfgr": 541, "ss.part.category": 542, "ss.part.brand": 543,
    # query stream (arrival times and template draws)
    "ss.queries": 590,
}


def mix64(z):
    """SplitMix64 output function on a uint64 array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> _U64(30))) * _M1
        z = (z ^ (z >> _U64(27))) * _M2
    return z ^ (z >> _U64(31))


def stream_base(seed: int, stream: int) -> np.uint64:
    s = mix64(np.array([stream], dtype=np.uint64))[0]
    return mix64(np.array([np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ s], dtype=np.uint64))[0]


def words(seed: int, stream: int, idx) -> np.ndarray:
    """64-bit words of (seed, stream) at the given int64 indices."""
    base = stream_base(seed, stream)
    i = np.asarray(idx, dtype=np.int64).astype(np.uint64)
    with np.errstate(over="ignore"):
        return mix64(base + (i + _U64(1)) * GAMMA)


def _idx(start: int, n: int) -> np.ndarray:
    return np.arange(start, start + n, dtype=np.int64)


def uniform_i32_at(seed: int, stream: int, idx, lo: int, hi: int) -> np.ndarray:
    assert lo <= hi and hi - lo + 1 <= 1 << 32
    w = words(seed, stream, idx)
    span = np.uint64(hi - lo + 1)
    with np.errstate(over="ignore"):
        off = ((w >> _U64(32)) * span) >> _U64(32)
    return (off.astype(np.int64) + lo).astype(np.int32)


def uniform_i32(seed: int, stream: int, n: int, lo: int, hi: int, start: int = 0) -> np.ndarray:
    return uniform_i32_at(seed, stream, _idx(start, n), lo, hi)


def uniform_f32_at(seed: int, stream: int, idx) -> np.ndarray:
    w = words(seed, stream, idx)
    return ((w >> _U64(40)).astype(np.float64) * 2.0 ** -24).astype(np.float32)


def uniform_f32(seed: int, stream: int, n: int, start: int = 0) -> np.ndarray:
    return uniform_f32_at(seed, stream, _idx(start, n))


def bits_i32_at(seed: int, stream: int, idx) -> np.ndarray:
    w = words(seed, stream, idx)
    return (w >> _U64(32)).astype(np.uint32).view(np.int32)


def bits_i32(seed: int, stream: int, n: int, start: int = 0) -> np.ndarray:
    return bits_i32_at(seed, stream, _idx(start, n))


def _feistel_bits(n: int) -> int:
    k = max(2, int(n - 1).bit_length()) if n > 1 else 2
    return k + (k & 1)


def _feistel(x: np.ndarray, keys: np.ndarray, half: int) -> np.ndarray:
    mask = np.uint64((1 << half) - 1)
    h = np.uint64(half)
    left = x >> h
    right = x & mask
    with np.errstate(over="ignore"):
        for r in range(4):
            f = mix64(right + keys[r]) & mask
            left, right = right, left ^ f
    return (left << h) | right


def perm_at(seed: int, stream: int, n: int, idx) -> np.ndarray:
    """Element(s) ``idx`` of the seeded permutation of [0, n), as int64."""
    idx = np.asarray(idx, dtype=np.int64)
    if n <= 0:
        assert idx.size == 0
        return idx.copy()
    half = _feistel_bits(n) // 2
    keys = words(seed, stream, np.arange(4, dtype=np.int64))
    y = _feistel(idx.astype(np.uint64), keys, half)
    nn = np.uint64(n)
    out_of_range = y >= nn
    while out_of_range.any():
        y[out_of_range] = _feistel(y[out_of_range], keys, half)
        out_of_range = y >= nn
    return y.astype(np.int64)


def perm_i32(seed: int, stream: int, n: int, start: int = 0, count: int | None = None) -> np.ndarray:
    count = n - start if count is None else count
    return perm_at(seed, stream, n, _idx(start, count)).astype(np.int32)


# ---------------------------------------------------------------------------
# Workload shapes (inputs only).  Sizes and value ranges of each synthetic table.
# ---------------------------------------------------------------------------

Q1_DIM_ROWS = 2556          # date-like dimension: 7 x 365 + 1 rows
Q1_YEARS = 7


def q1_tables(seed: int, n_fact: int) -> dict:
    """Fused filter-probe-aggregate workload: fact (fk, a, b, c), dimension (key, yr).

    fk ~ U[0, 2556), a ~ U[1, 50], b ~ U[0, 10], c ~ U[1, 100000]; the dimension's keys
    are a seeded permutation of 0..2555 and the row at position j has yr = j mod 7.
    """
    fact = {
        "fk": uniform_i32(seed, STREAMS["q1.fk"], n_fact, 0, Q1_DIM_ROWS - 1),
        "a": uniform_i32(seed, STREAMS["q1.a"], n_fact, 1, 50),
        "b": uniform_i32(seed, STREAMS["q1.b"], n_fact, 0, 10),
        "c": uniform_i32(seed, STREAMS["q1.c"], n_fact, 1, 100000),
    }
    dim = {
        "key": perm_i32(seed, STREAMS["q1.dim_key"], Q1_DIM_ROWS),
        "yr": (np.arange(Q1_DIM_ROWS) % Q1_YEARS).astype(np.int32),
    }
    return {"fact": fact, "dim": dim}


def select_threshold(sigma: float) -> int:
    """Inclusive upper bound ``hi`` for ``x < v`` with ``v = round(sigma * 2^31)``.

    Computed in Python integers so that sigma = 1 gives hi = 2^31 - 1 without
    overflowing int32 and sigma = 0 gives hi = -1 (no x in [0, 2^31) qualifies).
    """
    v = int(round(sigma * (1 << 31)))
    return min(v - 1, (1 << 31) - 1)


# Served star schema: dimension cardinalities and attribute domains.
SS_DIMS = {
    "date": {"rows": 2556, "fk": "fk_date", "attrs": {"year": 7, "month": 12}},
    "supp": {"rows": 200_000, "fk": "fk_supp", "attrs": {"region": 5, "nation": 25, "city": 250}},
    "cust": {"rows": 3_000_000, "fk": "fk_cust", "attrs": {"region": 5, "nation": 25, "city": 250}},
    "part": {"rows": 1_400_000, "fk": "fk_part", "attrs": {"mfgr": 5, "category": 25, "brand": 1000}},
}
SS_FACT_COLS = ["fk_date", "fk_supp", "fk_cust", "fk_part", "qty", "disc", "price", "cost"]
SS_FACT_RANGES = {
    "fk_date": (0, 2556 - 1), "fk_supp": (0, 200_000 - 1), "fk_cust": (0, 3_000_000 - 1),
    "fk_part": (0, 1_400_000 - 1), "qty": (1, 50), "disc": (0, 10), "price": (1, 100_000),
    "cost": (1, 60_000),
}


def ss_dim_scale(rows: int, scale: float) -> int:
    return max(1, int(round(rows * scale)))


def ss_fact_col(seed: int, name: str, n: int, start: int = 0, dim_scale: float = 1.0) -> np.ndarray:
    lo, hi = SS_FACT_RANGES[name]
    if name.startswith("fk_"):
        dim = {"fk_date": "date", "fk_supp": "supp", "fk_cust": "cust", "fk_part": "part"}[name]
        hi = ss_dim_scale(SS_DIMS[dim]["rows"], dim_scale) - 1
    return uniform_i32(seed, STREAMS["ss." + name], n, lo, hi, start)


def ss_dimension(seed: int, dim: str, dim_scale: float = 1.0) -> dict:
    spec = SS_DIMS[dim]
    rows = ss_dim_scale(spec["rows"], dim_scale)
    out = {"key": perm_i32(seed, STREAMS[f"ss.{dim}.key"], rows)}
    for attr, card in spec["attrs"].items():
        out[attr] = uniform_i32(seed, STREAMS[f"ss.{dim}.{attr}"], rows, 0, card - 1)
    return out


def ss_tables(seed: int, n_fact: int, dim_scale: float = 1.0) -> dict:
    """Host copy of the served star schema (used for small scales and oracle samples)."""
    fact = {c: ss_fact_col(seed, c, n_fact, 0, dim_scale) for c in SS_FACT_COLS}
    dims = {d: ss_dimension(seed, d, dim_scale) for d in SS_DIMS}
    return {"fact": fact, "dims": dims}


# Query templates of the served stream.  A query is a plain dict:
#   {"id": int, "arrival_s": float,
#    "fact_preds": [(col, lo, hi), ...],
#    "joins": [{"dim": d, "filters": [(attr, lo, hi), ...], "group": attr | None}, ...],
#    "agg": (op, col_a, col_b | None)}          op in {"sum", "mul", "sub", "add"}
SS_AGGS = [("mul", "price", "disc"), ("sum", "price", None), ("sub", "price", "cost")]
SS_GROUP_LIMIT = 10_000


def _draw(seed: int, qid: int, slot: int, lo: int, hi: int) -> int:
    return int(uniform_i32_at(seed, STREAMS["ss.queries"], [qid * 64 + slot], lo, hi)[0])


def _draw_unit(seed: int, qid: int, slot: int) -> float:
    return float(uniform_f32_at(seed, STREAMS["ss.queries"], [qid * 64 + slot])[0])


def ss_query(seed: int, qid: int) -> dict:
    """Query ``qid`` of the seeded stream: 1-4 joins, ranges chosen so that the product
    of per-predicate selectivities is log-uniform in [1e-4, 0.5], group-by attributes
    whose cardinality product is at most 10^4, and one of three SUM expressions."""
    dims = list(SS_DIMS)
    k = _draw(seed, qid, 0, 1, 4)
    # choose k distinct dimensions by a seeded partial Fisher-Yates over the 4 names
    order = dims[:]
    for i in range(k):
        j = _draw(seed, qid, 1 + i, i, len(order) - 1)
        order[i], order[j] = order[j], order[i]
    chosen = order[:k]
    target = 10 ** (np.log10(1e-4) + _draw_unit(seed, qid, 8) * (np.log10(0.5) - np.log10(1e-4)))
    per_dim = target ** (1.0 / k)
    joins = []
    groups = 1
    slot = 10
    for d in chosen:
        attrs = SS_DIMS[d]["attrs"]
        names = list(attrs)
        fattr = names[_draw(seed, qid, slot, 0, len(names) - 1)]
        card = attrs[fattr]
        width = max(1, min(card, int(round(per_dim * card))))
        lo = _draw(seed, qid, slot + 1, 0, card - width)
        filters = [(fattr, lo, lo + width - 1)] if width < card else []
        gattr = None
        gi = _draw(seed, qid, slot + 2, -1, len(names) - 1)
        if gi >= 0:
            gcard = attrs[names[gi]]
            if groups * gcard <= SS_GROUP_LIMIT:
                gattr = names[gi]
                groups *= gcard
        joins.append({"dim": d, "filters": filters, "group": gattr})
        slot += 3
    fact_preds = []
    if _draw(seed, qid, 30, 0, 3) == 0:      # a quarter of the queries also filter the fact table
        lo = _draw(seed, qid, 31, 1, 25)
        fact_preds.append(("qty", lo, lo + 24))
    agg = SS_AGGS[_draw(seed, qid, 40, 0, len(SS_AGGS) - 1)]
    return {"id": qid, "fact_preds": fact_preds, "joins": joins, "agg": agg}


def ss_arrivals(seed: int, n: int, rate_qps: float) -> np.ndarray:
    """Poisson arrival times (seconds) of n queries at ``rate_qps``: cumulative sums of
    exponential gaps -ln(1 - u) / rate with u from the query stream's words."""
    u = uniform_f32_at(seed, STREAMS["ss.queries"], np.arange(n, dtype=np.int64) * 64 + 63)
    gaps = -np.log1p(-u.astype(np.float64)) / rate_qps
    return np.cumsum(gaps)


def ss_group_count(query: dict) -> int:
    g = 1
    for j in query["joins"]:
        if j["group"] is not None:
            g *= SS_DIMS[j["dim"]]["attrs"][j["group"]]
    return g
