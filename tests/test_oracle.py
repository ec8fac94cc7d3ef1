"""Pins of the oracle against what the paper and the mathematics fix.

Each test checks the C oracle against something other than itself: the paper's worked
example, closed forms, exact rational arithmetic, invariants, textbook special cases,
or brute force (nested loops) on tiny inputs.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import datagen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
I32_MIN, I32_MAX = -(1 << 31), (1 << 31) - 1


def _golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split(":", 1)
                out[k.strip()] = [int(t) for t in v.split()]
    return out


# ------------------------------------------------------------------ selection

def test_tile_example_from_paper(orc):
    g = _golden("tile_example.txt")
    vals = np.array(g["values"], np.int32)
    flags = vals > g["predicate_gt"][0]
    counts, offsets, total, order = orc.tile_scan(flags, g["threads"][0], g["items_per_thread"][0])
    assert list(counts) == g["counts"]
    assert list(offsets) == g["offsets"]
    assert total == g["total"][0]
    # each thread's matches land in its own range, in its own item order
    for t in range(4):
        seg = order[offsets[t]: offsets[t] + counts[t]]
        assert all(i % 4 == t for i in seg) and list(seg) == sorted(seg)
    assert sorted(order) == [i for i in range(16) if flags[i]]
    # the selection over the same 16 values keeps exactly those 10 entries
    out = orc.select(vals, g["predicate_gt"][0] + 1, I32_MAX)
    assert out.size == g["total"][0]


@pytest.mark.parametrize("seed", range(6))
def test_select_brute_force(orc, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(0, 300))
    x = rng.integers(-50, 50, size=n).astype(np.int32)
    lo, hi = sorted(int(v) for v in rng.integers(-60, 60, size=2))
    expect = [v for v in x.tolist() if lo <= v <= hi]
    assert orc.select(x, lo, hi).tolist() == expect
    assert orc.select(x, hi + 1, lo).size == (0 if hi + 1 > lo else sum(1 for v in x if hi + 1 <= v <= lo))


def test_select_closed_form_on_permutation(orc):
    # x a permutation of 0..N-1: "x < v" keeps exactly v rows, namely 0..v-1, in the
    # order in which they occur in x.
    n = 50_000
    x = datagen.perm_i32(1, 2, n)
    for v in [0, 1, 7, 12_345, n - 1, n]:
        out = orc.select(x, I32_MIN, v - 1) if v > 0 else orc.select(x, 0, -1)
        assert out.size == v
        assert np.array_equal(np.sort(out), np.arange(v))
        assert np.array_equal(out, x[x < v])


def test_select_selectivity_edges(orc):
    x = datagen.uniform_i32(3, datagen.STREAMS["sel.x"], 100_000, 0, I32_MAX)
    assert orc.select(x, I32_MIN, datagen.select_threshold(0.0)).size == 0
    assert np.array_equal(orc.select(x, I32_MIN, datagen.select_threshold(1.0)), x)
    assert orc.select(x, I32_MIN, I32_MAX).size == x.size
    assert orc.select(np.array([I32_MIN, I32_MAX], np.int32), I32_MAX, I32_MAX).tolist() == [I32_MAX]


def test_select_threads_identical(orc):
    x = datagen.uniform_i32(3, 4, 123_457, -1000, 1000)
    a = orc.select(x, -10, 500)
    for t in (2, 3, 7):
        assert np.array_equal(orc.select(x, -10, 500, threads=t), a)


# ------------------------------------------------------------------ projection

def test_project_closed_forms(orc):
    x1 = np.array([0.0, 0.5, 0.25, 1.0, 0.125], np.float32)
    x2 = np.array([0.0, 0.25, 0.5, 1.0, 0.0625], np.float32)
    y = orc.project(x1, x2, 2.0, 3.0, 0)
    assert y.tolist() == [0.0, 1.75, 2.0, 5.0, 0.4375]
    s = orc.project(x1[:1], x2[:1], 2.0, 3.0, 1)
    assert s[0] == np.float32(0.5)          # sigmoid(0) = 1/2 exactly


def test_project_linear_is_correctly_rounded(orc):
    # Exact rational value of a*x1 + b*x2, rounded once to float32.
    x1 = datagen.uniform_f32(5, datagen.STREAMS["proj.x1"], 2000)
    x2 = datagen.uniform_f32(5, datagen.STREAMS["proj.x2"], 2000)
    y = orc.project(x1, x2, 2.0, 3.0, 0)
    for i in range(x1.size):
        exact = Fraction(float(x1[i])) * 2 + Fraction(float(x2[i])) * 3
        assert y[i] == np.float32(float(exact)), i


def test_project_sigmoid_against_high_precision(orc):
    # 1/(1+e^-y) evaluated in 50-digit decimal arithmetic from the exact rational y,
    # compared within one float32 ulp of the true value.
    from decimal import Decimal, getcontext
    getcontext().prec = 50
    x1 = datagen.uniform_f32(6, 1, 200)
    x2 = datagen.uniform_f32(6, 2, 200)
    for a, b in [(2.0, 3.0), (-2.0, -3.0)]:
        y = orc.project(x1, x2, a, b, 1)
        for i in range(x1.size):
            lin = Decimal(float(x1[i])) * Decimal(a) + Decimal(float(x2[i])) * Decimal(b)
            ref = float(1 / (1 + (-lin).exp()))
            ulp = float(np.spacing(np.float32(ref)))
            assert abs(float(y[i]) - ref) <= ulp, (a, i)
    # symmetry sigma(-y) = 1 - sigma(y)
    yp = orc.project(x1, x2, 2.0, 3.0, 1).astype(np.float64)
    yn = orc.project(x1, x2, -2.0, -3.0, 1).astype(np.float64)
    assert np.all(np.abs(yp + yn - 1.0) <= 2 * np.spacing(np.float32(1.0)))


# ------------------------------------------------------------------ hash join

def _nested_loop_join(bk, bv, fk, pay):
    s, m = 0, 0
    for i in range(len(fk)):
        for j in range(len(bk)):
            if fk[i] == bk[j]:
                s += int(pay[i]) * int(bv[j])
                m += 1
    s &= (1 << 64) - 1
    return (s - (1 << 64) if s >= 1 << 63 else s), m


@pytest.mark.parametrize("seed", range(5))
def test_join_nested_loop(orc, seed):
    rng = np.random.default_rng(100 + seed)
    nb = int(rng.integers(0, 60))
    bk = rng.choice(np.arange(-200, 200), size=nb, replace=False).astype(np.int32)
    bv = rng.integers(-100, 100, size=nb).astype(np.int32)
    npb = int(rng.integers(0, 150))
    fk = rng.integers(-220, 220, size=npb).astype(np.int32)
    pay = rng.integers(-100, 100, size=npb).astype(np.int32)
    assert orc.join_sum(bk, bv, fk, pay) == _nested_loop_join(bk, bv, fk, pay)


def test_join_closed_forms(orc):
    n = 4096
    bk = datagen.perm_i32(2, 3, n)
    ones = np.ones(n, np.int32)
    fk = datagen.uniform_i32(2, 4, 10_000, 0, n - 1)
    pay = datagen.uniform_i32(2, 5, 10_000, 1, 100)
    # every probe key exists; with unit build values the sum is the payload total
    assert orc.join_sum(bk, ones, fk, pay) == (int(pay.astype(np.int64).sum()), 10_000)
    # keys outside the build side contribute nothing
    assert orc.join_sum(bk, ones, fk + n, pay) == (0, 0)
    # value = key: sum of payload * fk
    vals = bk.copy()
    assert orc.join_sum(bk, vals, fk, pay)[0] == int((pay.astype(np.int64) * fk).sum())


def test_join_wraps_mod_2_64(orc):
    bk = np.array([1], np.int32)
    bv = np.array([I32_MAX], np.int32)
    fk = np.ones(8, np.int32)
    pay = np.full(8, I32_MAX, np.int32)
    assert orc.join_sum(bk, bv, fk, pay) == _nested_loop_join(bk, bv, fk, pay)


def test_join_rejects_duplicate_build_keys(orc):
    with pytest.raises(ValueError):
        orc.join_sum(np.array([3, 3], np.int32), np.array([1, 2], np.int32),
                     np.array([3], np.int32), np.array([1], np.int32))


def test_join_threads_identical(orc):
    bk = datagen.perm_i32(9, 1, 10_000)
    bv = datagen.uniform_i32(9, 2, 10_000, 1, 100)
    fk = datagen.uniform_i32(9, 3, 100_001, 0, 12_000)
    pay = datagen.uniform_i32(9, 4, 100_001, 1, 100)
    assert orc.join_sum(bk, bv, fk, pay) == orc.join_sum(bk, bv, fk, pay, threads=5)


# ------------------------------------------------------------------ sort

@pytest.mark.parametrize("seed", range(4))
def test_sort_matches_stable_library_sort(orc, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(0, 500))
    keys = rng.integers(-20, 20, size=n).astype(np.int32)
    vals = np.arange(n, dtype=np.int32)
    ko, vo = orc.sort(keys, vals)
    order = sorted(range(n), key=lambda i: int(keys[i]))     # Python's sort is stable
    assert ko.tolist() == [int(keys[i]) for i in order]
    assert vo.tolist() == order


def test_sort_properties_full_range(orc):
    n = 200_000
    keys = datagen.bits_i32(4, datagen.STREAMS["sort.key"], n)
    keys[::1000] = keys[0]                  # force duplicates
    vals = np.arange(n, dtype=np.int32)
    ko, vo = orc.sort(keys, vals)
    assert np.all(ko[:-1] <= ko[1:])                          # ordered, signed
    assert np.array_equal(np.sort(vo), vals)                  # permutation of row ids
    assert np.array_equal(keys[vo], ko)                       # pairs kept together
    same = ko[:-1] == ko[1:]
    assert np.all(vo[:-1][same] < vo[1:][same])               # stable
    assert ko[0] < 0 < ko[-1]


def test_sort_reversed_closed_form(orc):
    n = 1000
    keys = np.arange(n - 1, -1, -1, dtype=np.int32) - 500
    ko, vo = orc.sort(keys, np.arange(n, dtype=np.int32))
    assert np.array_equal(ko, np.arange(n, dtype=np.int32) - 500)
    assert np.array_equal(vo, np.arange(n - 1, -1, -1, dtype=np.int32))


# ------------------------------------------------------------------ query plans

def _brute_plan(cols, preds, joins, agg):
    op, a, b = agg
    groups = 1
    for j in joins:
        if j["group"] is not None:
            groups *= j["card"]
    sums = [0] * groups
    counts = [0] * groups
    n = len(cols[0])
    for r in range(n):
        if not all(lo <= cols[c][r] <= hi for c, lo, hi in preds):
            continue
        ok, g = True, 0
        for j in joins:
            hit = [d for d in range(len(j["keys"])) if j["keys"][d] == cols[j["fk_col"]][r]]
            if not hit or not all(lo <= arr[hit[0]] <= hi for arr, lo, hi in j["preds"]):
                ok = False
                break
            if j["group"] is not None:
                g = g * j["card"] + int(j["group"][hit[0]])
        if not ok:
            continue
        va = int(cols[a][r])
        vb = int(cols[b][r]) if b is not None else 0
        v = {"sum": va, "mul": va * vb, "sub": va - vb, "add": va + vb}[op]
        sums[g] += v
        counts[g] += 1
    return sums, counts


def _tiny_star(rng, n_fact=300):
    dims = []
    for rows, card in [(13, 3), (29, 4), (7, 2)]:
        keys = rng.choice(np.arange(-40, 60), size=rows, replace=False).astype(np.int32)
        attr = rng.integers(0, card, size=rows).astype(np.int32)
        other = rng.integers(0, 5, size=rows).astype(np.int32)
        dims.append((keys, attr, other, card))
    cols = [rng.integers(-45, 65, size=n_fact).astype(np.int32) for _ in range(3)]  # fks
    cols += [rng.integers(-30, 30, size=n_fact).astype(np.int32) for _ in range(3)]  # measures
    return dims, cols


@pytest.mark.parametrize("seed", range(8))
def test_plan_brute_force(orc, seed):
    rng = np.random.default_rng(1000 + seed)
    dims, cols = _tiny_star(rng)
    nj = int(rng.integers(0, 4))
    joins = []
    for j in range(nj):
        keys, attr, other, card = dims[j]
        preds = [(other, int(rng.integers(0, 3)), int(rng.integers(2, 5)))] if rng.random() < 0.7 else []
        grouped = rng.random() < 0.6
        joins.append({"fk_col": j, "keys": keys, "preds": preds,
                      "group": attr if grouped else None, "card": card if grouped else 1})
    preds = [(int(rng.integers(3, 6)), -20, int(rng.integers(-5, 25)))] if rng.random() < 0.5 else []
    for op in ["sum", "mul", "sub", "add"]:
        agg = (op, 4, 5 if op != "sum" else None)
        sums, counts = orc.run_plan_raw(cols, preds, joins, agg)
        bs, bc = _brute_plan(cols, preds, joins, agg)
        assert sums.tolist() == bs and counts.tolist() == bc, op
        s2, c2 = orc.run_plan_raw(cols, preds, joins, agg, threads=3)
        assert np.array_equal(s2, sums) and np.array_equal(c2, counts)


def test_plan_group_invariants(orc):
    t = datagen.ss_tables(21, 50_000, dim_scale=0.01)
    q = {"id": 0, "fact_preds": [("qty", 5, 40)],
         "joins": [{"dim": "supp", "filters": [("region", 1, 3)], "group": "nation"},
                   {"dim": "date", "filters": [], "group": "year"}],
         "agg": ("sub", "price", "cost")}
    sums, counts = orc.ss_run(t, q)
    assert sums.size == 25 * 7
    flat = dict(q, joins=[dict(j, group=None) for j in q["joins"]])
    s1, c1 = orc.ss_run(t, flat)
    assert int(sums.sum()) == int(s1[0]) and int(counts.sum()) == int(c1[0])
    # grouping by year alone equals summing the (nation, year) table over nations
    by_year = dict(q, joins=[dict(q["joins"][0], group=None), q["joins"][1]])
    s2, c2 = orc.ss_run(t, by_year)
    assert np.array_equal(s2, sums.reshape(25, 7).sum(axis=0))
    assert np.array_equal(c2, counts.reshape(25, 7).sum(axis=0))


def test_plan_single_join_no_preds_is_full_sum(orc):
    # every fk exists and no predicate filters: SUM over all rows of price - cost
    t = datagen.ss_tables(22, 20_000, dim_scale=0.01)
    q = {"id": 0, "fact_preds": [], "joins": [{"dim": "cust", "filters": [], "group": None}],
         "agg": ("sub", "price", "cost")}
    s, c = orc.ss_run(t, q)
    f = t["fact"]
    assert int(s[0]) == int((f["price"].astype(np.int64) - f["cost"]).sum())
    assert int(c[0]) == 20_000


def test_q1_year_partition_invariant(orc):
    t = datagen.q1_tables(31, 200_000)
    f, d = t["fact"], t["dim"]
    per_year = [orc.q1_run(f, d, year=y) for y in range(7)]
    # the same query without the year predicate, computed directly from the definition
    m = (f["a"] < 25) & (f["b"] >= 1) & (f["b"] <= 3)
    total = int((f["c"][m].astype(np.int64) * f["b"][m]).sum())
    assert sum(per_year) == total
    assert orc.q1_run(f, d, year=7) == 0       # no dimension row has year code 7


def test_q1_brute_force_small(orc):
    t = datagen.q1_tables(32, 3000)
    f, d = t["fact"], t["dim"]
    yr_of_key = {int(k): int(y) for k, y in zip(d["key"], d["yr"])}
    expect = 0
    for i in range(f["fk"].size):
        if yr_of_key[int(f["fk"][i])] == 3 and f["a"][i] < 25 and 1 <= f["b"][i] <= 3:
            expect += int(f["c"][i]) * int(f["b"][i])
    assert orc.q1_run(f, d) == expect


def test_plan_rejects_bad_group_codes(orc):
    cols = [np.array([0, 1], np.int32), np.array([5, 6], np.int32)]
    joins = [{"fk_col": 0, "keys": np.array([0, 1], np.int32), "preds": [],
              "group": np.array([0, 9], np.int32), "card": 3}]
    with pytest.raises(ValueError):
        orc.run_plan_raw(cols, [], joins, ("sum", 1, None))


def _brute_served(t, q):
    """A served query evaluated row by row from its dict: dimension rows looked up by key,
    filters and group attributes read by name, group id mixed-radix with the first grouped
    join most significant, the SUM expression by its operand names."""
    fact, dims = t["fact"], t["dims"]
    by_key = {d: {int(k): r for r, k in enumerate(cols["key"])} for d, cols in dims.items()}
    grouped = [j for j in q["joins"] if j["group"] is not None]
    cards = [datagen.SS_DIMS[j["dim"]]["attrs"][j["group"]] for j in grouped]
    n_groups = int(np.prod(cards)) if cards else 1
    sums, counts = [0] * n_groups, [0] * n_groups
    op, a, b = q["agg"]
    for i in range(fact["qty"].size):
        if not all(lo <= int(fact[c][i]) <= hi for c, lo, hi in q["fact_preds"]):
            continue
        codes, ok = {}, True
        for j in q["joins"]:
            r = by_key[j["dim"]].get(int(fact[datagen.SS_DIMS[j["dim"]]["fk"]][i]))
            if r is None or not all(lo <= int(dims[j["dim"]][at][r]) <= hi for at, lo, hi in j["filters"]):
                ok = False
                break
            if j["group"] is not None:
                codes[id(j)] = int(dims[j["dim"]][j["group"]][r])
        if not ok:
            continue
        g = 0
        for j, card in zip(grouped, cards):
            g = g * card + codes[id(j)]
        x = int(fact[a][i])
        y = int(fact[b][i]) if b is not None else 0
        sums[g] += {"sum": x, "mul": x * y, "sub": x - y, "add": x + y}[op]
        counts[g] += 1
    return sums, counts


def test_served_query_brute_force(orc):
    # queries of the seeded stream on a small star schema, each computed from its dict
    t = datagen.ss_tables(23, 4000, dim_scale=0.004)
    checked = 0
    for qid in range(60):
        q = datagen.ss_query(23, qid)
        bs, bc = _brute_served(t, q)
        s, c = orc.ss_run(t, q)
        assert s.tolist() == bs and c.tolist() == bc, q
        checked += sum(bc) > 0
    assert checked >= 10          # enough of them select rows for the comparison to bite
