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
    from paper_2003_01178_gb300.starschema import ResidentStarSchema, served_schema
    host = datagen.ss_tables(3, 500_009, dim_scale=0.02)
    fact = {k: torch.from_numpy(v).cuda() for k, v in host["fact"].items()}
    dims = {d: {k: torch.from_numpy(v).cuda() for k, v in t.items()} for d, t in host["dims"].items()}
    return host, ResidentStarSchema(served_schema(), fact, dims)


@pytest.mark.parametrize("realtime", [False, True])
def test_served_results_equal_alone_and_oracle(store, orc, realtime):
    from paper_2003_01178_gb300.server import QueryServer, one_at_a_time
    host, ss = store
    queries = [datagen.ss_query(21, q) for q in range(48)]
    arrivals = datagen.ss_arrivals(21, len(queries), 2000.0)
    server = QueryServer(ss, segments=5, max_slots=12, memory_budget=1 << 30)
    reqs, stats = server.serve(queries, arrivals, realtime=realtime)
    assert stats.completed == len(queries) and stats.max_active <= 12
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
