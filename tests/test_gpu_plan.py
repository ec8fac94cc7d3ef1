"""GPU parity of the fused select-join-aggregate kernels (one query, and the shared scan
of several queries) against the oracle, through the C ABI."""
import numpy as np
import pytest

import datagen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

I32_MIN = -(1 << 31)


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


def _q1_gpu(crys, fact, dim, year=3, kind=0):
    # kind 0: multiplicative hashing with linear probing; 2: a direct table (the dense date
    # keys' perfect hashing)
    cap = dim["key"].numel() if kind == crys.HASH_DIRECT else None
    ht = crys.HashTable.build(dim["key"], dim["yr"], filters=[(dim["yr"], year, year)], capacity=cap, kind=kind)
    sums, counts = crys.run_plan([fact["fk"], fact["a"], fact["b"], fact["c"]],
                                 [(1, I32_MIN, 24), (2, 1, 3)], [(0, ht, 0)], ("mul", 3, 2))
    return int(sums[0].item()), int(counts[0].item())


@pytest.mark.parametrize("n", [0, 1, 5, 1023, 4096, 4099, 100_003, 1 << 22, (1 << 24) + 3])
@pytest.mark.parametrize("variant", range(4))
@pytest.mark.parametrize("kind", [0, 2])
def test_q1_parity(crys, orc, n, variant, kind):
    crys.crys_set_tile(crys.OP_PLAN, variant)
    host = datagen.q1_tables(40 + n % 7, n)
    fact = {k: _dev(v) for k, v in host["fact"].items()}
    dim = {k: _dev(v) for k, v in host["dim"].items()}
    s, c = _q1_gpu(crys, fact, dim, kind=kind)
    assert s == orc.q1_run(host["fact"], host["dim"])
    crys.crys_set_tile(crys.OP_PLAN, 0)


@pytest.mark.parametrize("variant", range(4))
def test_selective_aggregate_loads(crys, orc, variant):
    """Filters that keep very few rows: the aggregate column is read only for the 16-byte
    groups with a live row (and stops being prefetched); sums stay exact."""
    crys.crys_set_tile(crys.OP_PLAN, variant)
    n = 3_000_017
    host = datagen.q1_tables(55, n)
    fact = {k: _dev(v) for k, v in host["fact"].items()}
    dim = {k: _dev(v) for k, v in host["dim"].items()}
    ht = crys.HashTable.build(dim["key"], dim["yr"], filters=[(dim["yr"], 3, 3)])
    cols = [fact["fk"], fact["a"], fact["b"], fact["c"]]
    hcols = [host["fact"][k] for k in ("fk", "a", "b", "c")]
    ojoin = [{"fk_col": 0, "keys": host["dim"]["key"], "preds": [(host["dim"]["yr"], 3, 3)], "group": None,
              "card": 1}]
    for preds, agg in [([(1, 1, 1), (2, 1, 3)], ("mul", 3, 2)), ([(1, 50, 50)], ("sum", 3, None)),
                       ([], ("sub", 3, 1)), ([(2, 10, 10)], ("add", 3, 3))]:
        sums, counts = crys.run_plan(cols, preds, [(0, ht, 0)], agg)
        rs, rc = orc.run_plan_raw(hcols, preds, ojoin, agg)
        assert int(sums[0].item()) == int(rs[0]) and int(counts[0].item()) == int(rc[0]), (preds, agg)
    crys.crys_set_tile(crys.OP_PLAN, 0)


@pytest.mark.parametrize("n", [1, 4099, 1_000_003, (1 << 22) + 5])
@pytest.mark.parametrize("variant", range(4))
def test_fixed_shape_plans(crys, orc, n, variant):
    """Plans of the Q1 family (one or two fact predicates, one join on a direct table with
    one or two field predicates, one group, SUM(a * b) or SUM(a)) run in the kernel
    compiled for their shape when a launch is short; exact against the oracle, ragged
    tails included."""
    crys.crys_set_tile(crys.OP_PLAN, variant)
    host = datagen.q1_tables(91 + n % 5, n)
    keys, yr = host["dim"]["key"], host["dim"]["yr"]
    mo = (np.arange(keys.size) % 12).astype(np.int32)
    packed = (yr | (mo << 3)).astype(np.int32)
    ht = crys.HashTable.build(_dev(keys), _dev(packed), capacity=keys.size, kind=crys.HASH_DIRECT)
    fact = {k: _dev(v) for k, v in host["fact"].items()}
    cols = [fact["fk"], fact["a"], fact["b"], fact["c"]]
    hcols = [host["fact"][k] for k in ("fk", "a", "b", "c")]
    for fps, opreds in [([(0, 3, 3, 3)], [(yr, 3, 3)]), ([(0, 3, 3, 3), (3, 4, 2, 5)], [(yr, 3, 3), (mo, 2, 5)])]:
        ojoin = [{"fk_col": 0, "keys": keys, "preds": opreds, "group": None, "card": 1}]
        for preds, agg in [([(1, I32_MIN, 24), (2, 1, 3)], ("mul", 3, 2)), ([(1, 10, 30)], ("mul", 3, 2)),
                           ([(2, 1, 3), (1, 5, 5)], ("sum", 3, None)), ([(1, 1, 40)], ("sum", 2, None))]:
            sums, counts = crys.run_plan(cols, preds, [(0, ht, 0, (0, 0), fps)], agg)
            rs, rc = orc.run_plan_raw(hcols, preds, ojoin, agg)
            assert int(sums[0].item()) == int(rs[0]) and int(counts[0].item()) == int(rc[0]), (n, fps, preds, agg)
    crys.crys_set_tile(crys.OP_PLAN, 0)


@pytest.mark.parametrize("variant", [2, 3])
def test_fixed_shape_selective_loads(crys, orc, variant):
    """Long launches with 4-row tiles: once a warp has seen that fewer than a third of the
    aggregate-only column's 128-byte lines are needed, it reads that column for live
    16-byte groups only; sums stay exact for sparse and dense plans alike."""
    crys.crys_set_tile(crys.OP_PLAN, variant)
    n = (1 << 25) + 3
    host = datagen.q1_tables(123, n)
    fact = {k: _dev(v) for k, v in host["fact"].items()}
    dim = {k: _dev(v) for k, v in host["dim"].items()}
    ht = crys.HashTable.build(dim["key"], dim["yr"], filters=[(dim["yr"], 3, 3)], capacity=dim["key"].numel(),
                              kind=crys.HASH_DIRECT)
    cols = [fact["fk"], fact["a"], fact["b"], fact["c"]]
    hcols = [host["fact"][k] for k in ("fk", "a", "b", "c")]
    ojoin = [{"fk_col": 0, "keys": host["dim"]["key"], "preds": [(host["dim"]["yr"], 3, 3)], "group": None,
              "card": 1}]
    for preds, agg in [([(1, 1, 1), (2, 1, 3)], ("mul", 3, 2)),   # 0.08% of rows: late column c read sparsely
                       ([(1, 1, 1)], ("mul", 3, 2)),               # two late columns (b, c)
                       ([(1, I32_MIN, 24), (2, 1, 3)], ("mul", 3, 2))]:  # the stated query (dense)
        sums, counts = crys.run_plan(cols, preds, [(0, ht, 0)], agg)
        rs, rc = orc.run_plan_raw(hcols, preds, ojoin, agg)
        assert int(sums[0].item()) == int(rs[0]) and int(counts[0].item()) == int(rc[0]), (preds, agg)
    crys.crys_set_tile(crys.OP_PLAN, 0)


def test_run_plan_in_cuda_graph(crys, orc):
    """A captured call (the output-clearing kernel, then the query kernel launched as its
    programmatic dependent) replays exactly, again and again."""
    n = 1_000_003
    host = datagen.q1_tables(7, n)
    fact = {k: _dev(v) for k, v in host["fact"].items()}
    dim = {k: _dev(v) for k, v in host["dim"].items()}
    ht = crys.HashTable.build(dim["key"], dim["yr"], filters=[(dim["yr"], 3, 3)], capacity=dim["key"].numel(),
                              kind=crys.HASH_DIRECT)
    table = crys.make_table([fact["fk"], fact["a"], fact["b"], fact["c"]])
    sums = torch.zeros(1, dtype=torch.int64, device="cuda")
    counts = torch.zeros(1, dtype=torch.int64, device="cuda")
    plan = crys.make_plan([(1, I32_MIN, 24), (2, 1, 3)], [(0, ht, 0)], ("mul", 3, 2), sums, counts)
    expect = orc.q1_run(host["fact"], host["dim"])
    crys.crys_run_plan(table, plan)  # attributes and caches outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        crys.crys_run_plan(table, plan, torch.cuda.current_stream())
    for _ in range(3):
        sums.fill_(-1)
        counts.fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        assert int(sums.item()) == expect


def test_q1_year_invariant_on_gpu(crys, orc):
    host = datagen.q1_tables(77, 1 << 20)
    fact = {k: _dev(v) for k, v in host["fact"].items()}
    dim = {k: _dev(v) for k, v in host["dim"].items()}
    per_year = [_q1_gpu(crys, fact, dim, y)[0] for y in range(7)]
    assert per_year == [orc.q1_run(host["fact"], host["dim"], y) for y in range(7)]


def _schema_tables(seed, n, scale):
    host = datagen.ss_tables(seed, n, dim_scale=scale)
    fact = {k: _dev(v) for k, v in host["fact"].items()}
    dims = {d: {k: _dev(v) for k, v in t.items()} for d, t in host["dims"].items()}
    return host, fact, dims


@pytest.fixture(scope="module")
def star(crys):
    from paper_2003_01178_gb300.starschema import ResidentStarSchema, Schema
    host, fact, dims = _schema_tables(5, 300_007, 0.02)
    return host, ResidentStarSchema(Schema.from_spec(datagen.SS_FACT_COLS, datagen.SS_DIMS), fact, dims)


def _check(orc, host, cq, query):
    rs, rc = orc.ss_run(host, query)
    assert np.array_equal(cq.sums.cpu().numpy(), rs), query
    assert np.array_equal(cq.counts.cpu().numpy(), rc), query


@pytest.mark.parametrize("mode", ["filtered", "resident"])
@pytest.mark.parametrize("variant", range(4))
def test_star_queries_one_at_a_time(crys, orc, star, variant, mode):
    crys.crys_set_tile(crys.OP_PLAN, variant)
    host, ss = star
    for qid in range(12):
        q = datagen.ss_query(9, qid + 100 * variant)
        cq = ss.compile(q, mode=mode)
        ss.run(cq)
        _check(orc, host, cq, q)
    crys.check_device_errors()
    crys.crys_set_tile(crys.OP_PLAN, 0)


@pytest.mark.parametrize("mode", ["filtered", "resident"])
@pytest.mark.parametrize("variant", range(4))
def test_shared_scan_equals_alone(crys, orc, star, variant, mode):
    # resident mode: one batch-wide probe per dimension; filtered mode: more than 8
    # distinct tables, so every join probes for its own query
    crys.crys_set_tile(crys.OP_SHARED_SCAN, variant)
    host, ss = star
    queries = [datagen.ss_query(13, qid) for qid in range(20)]
    mix = [ss.compile(q, mode=mode) for q in queries]
    ss.run_shared(mix)
    for cq, q in zip(mix, queries):
        alone = ss.compile(q, mode="filtered")
        ss.run(alone)
        assert torch.equal(alone.sums, cq.sums) and torch.equal(alone.counts, cq.counts)
        _check(orc, host, cq, q)
    crys.check_device_errors()
    crys.crys_set_tile(crys.OP_SHARED_SCAN, 0)


def test_packed_fields(crys):
    n = 100_003
    a = torch.from_numpy(datagen.uniform_i32(1, 1, n, 0, 6)).cuda()
    b = torch.from_numpy(datagen.uniform_i32(1, 2, n, 0, 999)).cuda()
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    crys.crys_pack_fields([a, b], [0, 3], [3, 10], n, out)
    assert torch.equal(out, a | (b << 3))
    with pytest.raises(crys.CrystalError):
        crys.crys_pack_fields([a, b], [0, 2], [3, 10], n, out)   # overlapping fields


def test_shared_scan_segments_accumulate(crys, orc, star):
    host, ss = star
    queries = [datagen.ss_query(14, qid) for qid in range(32)]
    mix = [ss.compile(q, mode="resident") for q in queries]
    n = ss.n_rows
    cuts = [0, 4096, 65_536, 65_540, 200_000, n]
    for i, (a, b) in enumerate(zip(cuts[:-1], cuts[1:])):
        ss.run_shared(mix, a, b, accumulate=i > 0)
    for cq, q in zip(mix, queries):
        _check(orc, host, cq, q)


def test_group_accumulator_modes(crys, orc, star):
    # G = 1 (registers), small G (shared memory) and G = 25 * 1000 * 7 = 175000 groups,
    # beyond the shared-memory budget (global atomics), must all agree with the oracle.
    host, ss = star
    qs = [
        {"id": 0, "fact_preds": [], "joins": [{"dim": "date", "filters": [], "group": None}],
         "agg": ("sum", "price", None)},
        {"id": 1, "fact_preds": [("disc", 1, 3)],
         "joins": [{"dim": "supp", "filters": [("region", 0, 2)], "group": "nation"},
                   {"dim": "date", "filters": [], "group": "year"}], "agg": ("mul", "price", "disc")},
        {"id": 2, "fact_preds": [],
         "joins": [{"dim": "cust", "filters": [], "group": "nation"},
                   {"dim": "part", "filters": [("mfgr", 1, 3)], "group": "brand"},
                   {"dim": "date", "filters": [], "group": "year"}], "agg": ("sub", "price", "cost")},
    ]
    for mode in ("filtered", "resident"):
        for q in qs:
            cq = ss.compile(q, mode=mode)
            ss.run(cq)
            _check(orc, host, cq, q)
        mix = [ss.compile(q, mode=mode) for q in qs]
        ss.run_shared(mix)
        for cq, q in zip(mix, qs):
            _check(orc, host, cq, q)
