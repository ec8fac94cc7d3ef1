"""GPU parity of the shared scan with query bitmaps (crys_run_plans_tagged) on direct
dimension tables: against the oracle and against each plan run alone, for the cases the
bitmaps must get right: two joins of one query through the same (column, table) pair,
one table joined through two fact columns, foreign keys outside the table, a query no
row can satisfy, more than two fact predicates, a query without joins, group counts
beyond the shared-memory accumulators, row segments, every tile shape, and a batch that
cannot be tagged (falls back to the plain shared scan)."""
import numpy as np
import pytest

import datagen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def crys():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2003_01178_gb300 import _build
    _build.build()
    import paper_2003_01178_gb300 as crys
    crys.crys_device_errors(clear=True)
    yield crys
    assert crys.crys_device_errors(clear=True) == 0
    for op in range(crys.NUM_OPS):
        crys.crys_set_tile(op, 0)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


N = 150_003
ND0, ND1 = 1000, 64


@pytest.fixture(scope="module")
def world(crys):
    s = 21
    fact = [datagen.uniform_i32(s, 1, N, -3, ND0 + 40),   # 0: fk into D0, some outside
            datagen.uniform_i32(s, 2, N, 0, ND1 - 1),     # 1: fk into D1 (also valid D0 keys)
            datagen.uniform_i32(s, 3, N, 1, 50),          # 2: a
            datagen.uniform_i32(s, 4, N, 0, 10),          # 3: b
            datagen.uniform_i32(s, 5, N, 1, 100_000)]     # 4: c
    d0 = {"key": datagen.perm_i32(s, 6, ND0), "x": datagen.uniform_i32(s, 7, ND0, 0, 15),
          "y": datagen.uniform_i32(s, 8, ND0, 0, 99)}
    d1 = {"key": datagen.perm_i32(s, 9, ND1), "z": datagen.uniform_i32(s, 10, ND1, 0, 7)}
    p0 = _dev(d0["x"] | (d0["y"] << 4))                 # x: bits 0-3, y: bits 4-10
    p1 = _dev(d1["z"])                                  # z: bits 0-2
    t0 = crys.HashTable.build(_dev(d0["key"]), p0, kind=crys.HASH_DIRECT)
    t1 = crys.HashTable.build(_dev(d1["key"]), p1, kind=crys.HASH_DIRECT)
    cols = [_dev(c) for c in fact]
    return {"fact": fact, "cols": cols, "table": crys.make_table(cols), "d0": d0, "d1": d1,
            "t0": t0, "t1": t1}


X, Y, Z = (0, 4), (4, 7), (0, 3)   # (shift, bits) of the packed fields


def _queries(w):
    """(gpu joins, oracle joins, fact preds, agg) per query."""
    d0, d1, t0, t1 = w["d0"], w["d1"], w["t0"], w["t1"]

    def j0(fk, card=0, group=None, fps=(), ofps=()):
        g = {"x": X, "y": Y}[group] if group else (0, 0)
        return ((fk, t0, card, g, list(fps)),
                {"fk_col": fk, "keys": d0["key"], "preds": list(ofps),
                 "group": d0[group] if group else None, "card": card or 1})

    def j1(fk, card=0, fps=(), ofps=()):
        return ((fk, t1, card, Z if card else (0, 0), list(fps)),
                {"fk_col": fk, "keys": d1["key"], "preds": list(ofps),
                 "group": d1["z"] if card else None, "card": card or 1})

    qs = [
        # one join, a filter and a 100-way grouping
        ([j0(0, 100, "y", [(*X, 2, 9)], [(d0["x"], 2, 9)])], [], ("sum", 4, None)),
        # two joins through the same pair, grouped by the second
        ([j0(0, 0, None, [(*X, 0, 7)], [(d0["x"], 0, 7)]),
          j0(0, 16, "x", [(*Y, 10, 60)], [(d0["y"], 10, 60)])], [], ("mul", 4, 3)),
        # the same table joined through two fact columns (two pairs)
        ([j0(0, 16, "x"), j0(1, 0, None, [(*Y, 0, 30)], [(d0["y"], 0, 30)])], [], ("sub", 4, 2)),
        # three fact predicates and a one-row dimension filter
        ([j1(1, 0, [(*Z, 3, 3)], [(d1["z"], 3, 3)])], [(2, 10, 40), (3, 1, 9), (4, 100, 90_000)],
         ("add", 4, 3)),
        # no row can qualify
        ([j0(0, 16, "x")], [(2, 5, 4)], ("sum", 2, None)),
        # no joins at all
        ([], [(3, 2, 2)], ("sum", 4, None)),
        # 100 * 16 * 8 groups: beyond the shared-memory accumulators
        ([j0(0, 100, "y"), j0(0, 16, "x"), j1(1, 8)], [], ("mul", 2, 3)),
        # two predicates on one field, an empty one (lo > hi) on another
        ([j0(0, 0, None, [(*X, 3, 12), (*Y, 50, 40)], [(d0["x"], 3, 12), (d0["y"], 50, 40)])], [],
         ("sum", 4, None)),
    ]
    rng = np.random.default_rng(3)
    while len(qs) < 32:
        lo = int(rng.integers(0, 12))
        hi = lo + int(rng.integers(0, 6))
        zl = int(rng.integers(0, 8))
        qs.append(([j0(0, 16 if len(qs) % 2 else 0, "x" if len(qs) % 2 else None,
                       [(*X, lo, hi)], [(d0["x"], lo, hi)]),
                    j1(1, 8 if len(qs) % 3 == 0 else 0, [(*Z, zl, 7)], [(d1["z"], zl, 7)])],
                   [(2, int(rng.integers(1, 20)), 50)], ("mul", 4, 2)))
    return qs


def _plans(crys, qs):
    plans, outs = [], []
    for joins, preds, agg in qs:
        g = crys.plan_groups([j for j, _ in joins])
        s = torch.zeros(g, dtype=torch.int64, device="cuda")
        c = torch.zeros(g, dtype=torch.int64, device="cuda")
        plans.append(crys.make_plan(preds, [j for j, _ in joins], agg, s, c))
        outs.append((s, c))
    return plans, outs


def _tagged(crys, w, plans, segments=((0, N),)):
    need = crys.crys_run_plans_tagged_bytes(w["table"], plans)
    scratch = torch.empty(max(need, 16), dtype=torch.uint8, device="cuda")
    for i, (a, b) in enumerate(segments):
        crys.crys_run_plans_tagged(w["table"], plans, a, b, crys.ACCUMULATE if i else 0, scratch, need)
    return need


@pytest.mark.parametrize("variant", range(4))
def test_tagged_matches_oracle_and_alone(crys, orc, world, variant):
    crys.crys_set_tile(crys.OP_TAGGED_SCAN, variant)
    qs = _queries(world)
    plans, outs = _plans(crys, qs)
    assert _tagged(crys, world, plans) > 0
    alone_plans, alone = _plans(crys, qs)
    for p in alone_plans:
        crys.crys_run_plan(world["table"], p)
    for (joins, preds, agg), (s, c), (sa, ca) in zip(qs, outs, alone):
        rs, rc = orc.run_plan_raw(world["fact"], preds, [o for _, o in joins], agg)
        assert np.array_equal(s.cpu().numpy(), rs) and np.array_equal(c.cpu().numpy(), rc)
        assert torch.equal(s, sa) and torch.equal(c, ca)
    crys.check_device_errors()
    crys.crys_set_tile(crys.OP_TAGGED_SCAN, 0)


def test_tagged_segments_and_small_batches(crys, orc, world):
    qs = _queries(world)
    for batch in (qs[:1], qs[3:6], qs):
        plans, outs = _plans(crys, batch)
        _tagged(crys, world, plans, [(0, 4), (4, 4100), (4100, 4100), (4100, 77_776), (77_776, N)])
        for (joins, preds, agg), (s, c) in zip(batch, outs):
            rs, rc = orc.run_plan_raw(world["fact"], preds, [o for _, o in joins], agg)
            assert np.array_equal(s.cpu().numpy(), rs) and np.array_equal(c.cpu().numpy(), rc)


def test_untaggable_batch_falls_back(crys, orc, world):
    # a join on a multiplicative-hash table: no bitmaps (0 bytes), same results
    d1 = world["d1"]
    tm = crys.HashTable.build(_dev(d1["key"]), _dev(d1["z"]))
    qs = _queries(world)[:4]
    plans, outs = _plans(crys, qs)
    s = torch.zeros(8, dtype=torch.int64, device="cuda")
    c = torch.zeros(8, dtype=torch.int64, device="cuda")
    plans.append(crys.make_plan([], [(1, tm, 8)], ("sum", 4, None), s, c))
    assert crys.crys_run_plans_tagged_bytes(world["table"], plans) == 0
    crys.crys_run_plans_tagged(world["table"], plans, 0, N, 0, None, 0)
    rs, rc = orc.run_plan_raw(world["fact"], [], [{"fk_col": 1, "keys": d1["key"], "preds": [],
                                                   "group": d1["z"], "card": 8}], ("sum", 4, None))
    assert np.array_equal(s.cpu().numpy(), rs) and np.array_equal(c.cpu().numpy(), rc)
    for (joins, preds, agg), (ss, cc) in zip(qs, outs):
        rs, rc = orc.run_plan_raw(world["fact"], preds, [o for _, o in joins], agg)
        assert np.array_equal(ss.cpu().numpy(), rs)


def test_tagged_every_row_expands_every_query(crys, orc, world):
    # 32 queries without dimension filters: every row expands 32 (row, query) pairs, so a
    # warp's round holds 1024 of them and goes through the list in several windows
    qs = []
    for i in range(32):
        joins = [] if i % 3 else [((0, world["t0"], 16, X, []),
                                   {"fk_col": 0, "keys": world["d0"]["key"], "preds": [],
                                    "group": world["d0"]["x"], "card": 16})]
        qs.append((joins, [(2, 1, 50 - i)], ("sum", 4, None) if i % 2 else ("mul", 4, 3)))
    plans, outs = _plans(crys, qs)
    _tagged(crys, world, plans)
    for (joins, preds, agg), (s, c) in zip(qs, outs):
        rs, rc = orc.run_plan_raw(world["fact"], preds, [o for _, o in joins], agg)
        assert np.array_equal(s.cpu().numpy(), rs) and np.array_equal(c.cpu().numpy(), rc)


@pytest.mark.parametrize("variant", [0, 2, 3])
def test_tagged_every_fact_column_finishes(crys, orc, world, variant):
    """Every fact column is read by some query's predicates or aggregate (foreign-key
    columns included), through all four (column, table) pairs, with more than two fact
    predicates: each column is staged beside the pairs' values and read back from there."""
    crys.crys_set_tile(crys.OP_TAGGED_SCAN, variant)
    d0, d1, t0, t1 = world["d0"], world["d1"], world["t0"], world["t1"]

    def j(fk, table, dim, field, card, name, fps=()):
        return ((fk, table, card, field if card else (0, 0), [(*field, lo, hi) for lo, hi in fps]),
                {"fk_col": fk, "keys": dim["key"], "preds": [(dim[name], lo, hi) for lo, hi in fps],
                 "group": dim[name] if card else None, "card": card or 1})

    qs = [
        ([j(0, t0, d0, X, 16, "x")], [(1, 0, 40)], ("sum", 0, None)),
        ([j(1, t0, d0, Y, 0, "y", [(0, 50)])], [(0, 0, 500), (3, 1, 9)], ("mul", 1, 3)),
        ([j(1, t1, d1, Z, 8, "z")], [(2, 5, 45), (3, 0, 8), (4, 10, 99_000), (0, -3, 900)], ("sub", 4, 2)),
        ([j(0, t1, d1, Z, 0, "z", [(1, 6)])], [], ("add", 0, 1)),
        ([j(0, t0, d0, Y, 0, "y", [(20, 80)]), j(1, t1, d1, Z, 8, "z")], [(4, 1, 50_000)], ("add", 3, 4)),
    ]
    plans, outs = _plans(crys, qs)
    assert _tagged(crys, world, plans) > 0
    for (joins, preds, agg), (s, c) in zip(qs, outs):
        rs, rc = orc.run_plan_raw(world["fact"], preds, [o for _, o in joins], agg)
        assert np.array_equal(s.cpu().numpy(), rs) and np.array_equal(c.cpu().numpy(), rc)
    crys.check_device_errors()
    crys.crys_set_tile(crys.OP_TAGGED_SCAN, 0)


_PRED_CASES = {
    # two columns of small range: folded into the bitmaps (one table per column); two
    # predicates of one query on one column, a range reaching below the column's values,
    # one no row passes (b <= 10), one no row can satisfy (lo > hi), and on b a union of
    # ranges 256 values wide
    "folded": [[(2, 10, 40), (2, 20, 60)], [(3, 1, 9)], [(2, -5, 3)], [(3, 11, 20)], [(2, 30, 20)],
               [(2, 1, 50), (3, 0, 10)], [(3, -235, 5)], []],
    # the same with three predicated columns: finishing tests them
    "three_columns": [[(2, 10, 40), (2, 20, 60)], [(3, 1, 9)], [(1, 0, 31)], [(2, 30, 20)], []],
    # a column whose predicates span 257 values: finishing tests them
    "wide": [[(0, 0, 256)], [(3, 1, 9)], [(2, 5, 45)], []],
}


@pytest.mark.parametrize("variant", [0, 2])
@pytest.mark.parametrize("case", sorted(_PRED_CASES))
def test_tagged_fact_predicates(crys, orc, world, variant, case):
    """Fact predicates in the bitmaps or in finishing, each query against the oracle."""
    crys.crys_set_tile(crys.OP_TAGGED_SCAN, variant)
    d0, t0 = world["d0"], world["t0"]
    qs = []
    for i, preds in enumerate(_PRED_CASES[case]):
        joins = [((0, t0, 16, X, []),
                  {"fk_col": 0, "keys": d0["key"], "preds": [], "group": d0["x"], "card": 16})] if i % 2 else []
        qs.append((joins, preds, ("mul", 4, 3) if i % 3 else ("sum", 4, None)))
    plans, outs = _plans(crys, qs)
    _tagged(crys, world, plans, [(0, 40_000), (40_000, N)])
    for (joins, preds, agg), (s, c) in zip(qs, outs):
        rs, rc = orc.run_plan_raw(world["fact"], preds, [o for _, o in joins], agg)
        assert np.array_equal(s.cpu().numpy(), rs) and np.array_equal(c.cpu().numpy(), rc)
    crys.check_device_errors()
    crys.crys_set_tile(crys.OP_TAGGED_SCAN, 0)
