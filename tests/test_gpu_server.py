"""The served stream: continuous batching gives every query the same result as running
it alone (bit-exact int64 sums and counts), and both equal the oracle."""
import numpy as np
import pytest

import datagen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def store():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2003_01178_gb300 import _build
    _build.build()
    from paper_2003_01178_gb300.starschema import ResidentStarSchema, Schema
    host = datagen.ss_tables(3, 500_009, dim_scale=0.02)
    fact = {k: torch.from_numpy(v).cuda() for k, v in host["fact"].items()}
    dims = {d: {k: torch.from_numpy(v).cuda() for k, v in t.items()} for d, t in host["dims"].items()}
    return host, ResidentStarSchema(Schema.from_spec(datagen.SS_FACT_COLS, datagen.SS_DIMS), fact, dims)


@pytest.mark.parametrize("graphs", [True, False])
@pytest.mark.parametrize("realtime", [False, True])
def test_served_results_equal_alone_and_oracle(store, orc, realtime, graphs):
    from paper_2003_01178_gb300.server import QueryServer, one_at_a_time
    host, ss = store
    queries = [datagen.ss_query(21, q) for q in range(48)]
    arrivals = datagen.ss_arrivals(21, len(queries), 2000.0)
    server = QueryServer(ss, segments=5, max_slots=12, memory_budget=1 << 30, graphs=graphs)
    reqs, stats = server.serve(queries, arrivals, realtime=realtime)
    assert stats.completed == len(queries) and stats.max_active <= 12
    # with graphs every launch is a replay of one of the two captured graphs
    assert stats.replays == (stats.launches if graphs else 0)
    alone, _ = one_at_a_time(ss, queries, arrivals, realtime=False)
    for r, a, q in zip(reqs, alone, queries):
        assert np.array_equal(r.result[0], a[0]) and np.array_equal(r.result[1], a[1])
        rs, rc = orc.ss_run(host, q)
        assert np.array_equal(r.result[0], rs) and np.array_equal(r.result[1], rc)
        assert r.latency_s >= 0


def test_memory_budget_limits_concurrency(store, orc):
    from paper_2003_01178_gb300.server import QueryServer
    host, ss = store
    queries = [datagen.ss_query(22, q) for q in range(16)]
    biggest = max(ss.memory_needed(q) for q in queries)
    server = QueryServer(ss, segments=3, max_slots=32, memory_budget=biggest)
    reqs, stats = server.serve(queries, np.zeros(len(queries)), realtime=False)
    assert stats.completed == 16 and stats.deferred > 0
    for r, q in zip(reqs, queries):
        rs, rc = orc.ss_run(host, q)
        assert np.array_equal(r.result[0], rs) and np.array_equal(r.result[1], rc)


def test_replayed_launch_equals_direct(store, orc):
    """The argument-block launch (copied from pinned memory, replayed from a graph) gives
    what the direct tagged scan gives, segment by segment, with outputs cleared by the
    first launch and re-tagging only when the batch changes."""
    import paper_2003_01178_gb300 as crys
    from paper_2003_01178_gb300.starschema import ReplayedScan
    host, ss = store
    queries = [datagen.ss_query(23, q) for q in range(20)]
    stream = torch.cuda.Stream()
    rep = ReplayedScan(ss, stream)
    with torch.cuda.stream(stream):
        mine = [ss.compile(q, zero=False) for q in queries]
        for c in mine:                                  # garbage that the first launch clears
            c.sums.fill_(12345)
            c.counts.fill_(-7)
    n = ss.n_rows
    cuts = [0, 4096, 200_000, n]
    assert rep.launch(mine[:12], cuts[0], cuts[1], list(range(12)))
    assert rep.launch(mine[:12], cuts[1], cuts[2], [])           # same batch: no re-tagging
    assert rep.launch(mine, cuts[2], cuts[3], list(range(12, 20)))  # batch grows
    assert rep.launch(mine[12:], cuts[0], cuts[2], [])
    stream.synchronize()
    assert rep.replays == 4
    for c, q in zip(mine, queries):
        rs, rc = orc.ss_run(host, q)
        assert np.array_equal(c.sums.cpu().numpy(), rs) and np.array_equal(c.counts.cpu().numpy(), rc)
    crys.check_device_errors()


def test_block_for_another_tile_shape_is_refused(store):
    """A block prepared for one tile shape and launched under another does no work and
    raises the bounds flag (the kernel checks the shape before touching shared memory)."""
    import paper_2003_01178_gb300 as crys
    host, ss = store
    cq = ss.compile(datagen.ss_query(24, 0))
    nb = crys.crys_tagged_block_bytes()
    hb = torch.empty(nb, dtype=torch.uint8, pin_memory=True)
    need = crys.crys_run_plans_tagged_bytes(ss.table, [cq.plan])
    scratch = ss.scratch(need)
    crys.crys_set_tile(crys.OP_TAGGED_SCAN, 0)
    assert crys.crys_tagged_prepare(ss.table, [cq.plan], 0, ss.n_rows, crys.TAG_ANNOTATE, [0], scratch,
                                    scratch.numel(), hb.data_ptr()) == crys.OK
    db = hb.cuda()
    before = cq.sums.clone()
    crys.crys_set_tile(crys.OP_TAGGED_SCAN, 2)           # another tile shape
    crys.crys_tagged_launch(db)
    torch.cuda.synchronize()
    crys.crys_set_tile(crys.OP_TAGGED_SCAN, 0)
    assert crys.crys_device_errors(clear=True) & crys.DEV_BOUNDS
    assert torch.equal(cq.sums, torch.zeros_like(before))   # cleared by the prepare kernel only


def test_replayed_scan_follows_a_new_tile_shape(store, orc):
    """Graphs captured under one tile shape are captured again when the shape changes
    (as the autotuner may do between launches); results stay exact."""
    import paper_2003_01178_gb300 as crys
    from paper_2003_01178_gb300.starschema import ReplayedScan
    host, ss = store
    queries = [datagen.ss_query(25, q) for q in range(10)]
    stream = torch.cuda.Stream()
    rep = ReplayedScan(ss, stream)
    with torch.cuda.stream(stream):
        mine = [ss.compile(q, zero=False) for q in queries]
    n = ss.n_rows
    try:
        crys.crys_set_tile(crys.OP_TAGGED_SCAN, 0)
        assert rep.launch(mine, 0, 100_000, list(range(10)))
        crys.crys_set_tile(crys.OP_TAGGED_SCAN, 2)      # two 512-thread blocks per SM
        assert rep.launch(mine, 100_000, 200_000, [])
        crys.crys_set_tile(crys.OP_TAGGED_SCAN, 1)
        assert rep.launch(mine, 200_000, n, [])
        stream.synchronize()
    finally:
        crys.crys_set_tile(crys.OP_TAGGED_SCAN, 0)
    assert crys.crys_device_errors(clear=True) == 0
    for c, q in zip(mine, queries):
        rs, rc = orc.ss_run(host, q)
        assert np.array_equal(c.sums.cpu().numpy(), rs) and np.array_equal(c.counts.cpu().numpy(), rc)
