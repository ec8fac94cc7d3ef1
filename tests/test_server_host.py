"""Host-side logic of the serving loop (no GPU): admission by slots and memory, requests
that can never fit, segment bounds of the circular scan."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2003_01178_gb300.server import QueryServer, Request  # noqa: E402


class FakeStore:
    def __init__(self, n_rows, need):
        self.n_rows = n_rows
        self.device = torch.device("cpu")
        self._need = need

    def memory_needed(self, query, mode="resident"):
        return self._need[query["id"]]


def _server(store, **kw):
    s = QueryServer.__new__(QueryServer)
    s.store, s.max_slots, s.memory_budget = store, kw.get("max_slots", 32), kw.get("budget", 1000)
    s.mode = "resident"
    n = store.n_rows
    step = -(-n // kw.get("segments", 8))
    step = (step + 4095) // 4096 * 4096
    s.bounds = [(b, min(n, b + step)) for b in range(0, n, step)] or [(0, 0)]
    s.next_segment = 0
    return s


def test_admission_by_memory_and_slots():
    store = FakeStore(1 << 20, {0: 400, 1: 500, 2: 200, 3: 1})
    s = _server(store, budget=1000, max_slots=3)
    reqs = s.prepare([{"id": i} for i in range(4)], [0, 0, 0, 0])
    active = []
    for r in reqs[:2]:
        assert s.fits(r, active)
        active.append(r)
    assert not s.fits(reqs[2], active)          # 400 + 500 + 200 > 1000
    assert s.fits(reqs[3], active)              # 901 <= 1000
    active.append(reqs[3])
    assert not s.fits(Request({"id": 9}, 0.0, mem=0), active)   # all 3 slots taken


def test_query_larger_than_budget_is_refused_up_front():
    store = FakeStore(1000, {0: 10, 1: 5000})
    s = _server(store, budget=1000)
    with pytest.raises(MemoryError):
        s.prepare([{"id": 0}, {"id": 1}], [0.0, 0.1])


def test_segments_cover_rows_once_and_stay_aligned():
    for n in (1, 4095, 4096, 4097, 10_000_000, 600_000_000):
        s = _server(FakeStore(n, {}), segments=8)
        assert s.bounds[0][0] == 0 and s.bounds[-1][1] == n
        for (a, b), (c, _) in zip(s.bounds, s.bounds[1:]):
            assert b == c and a % 4096 == 0
        assert len(s.bounds) <= 8


class _Event:
    def synchronize(self):
        pass


class _HostServer(QueryServer):
    """The serving loop with its device steps replaced by host bookkeeping: each launch
    checks that the queries still holding memory (admitted and not yet harvested) fit the
    budget."""

    def __init__(self, store, budget, max_slots, segments):
        srv = _server(store, budget=budget, max_slots=max_slots, segments=segments)
        self.__dict__.update(srv.__dict__)
        self.replay = None
        self.h2d_bytes = 0
        self.requests = []
        self.worst = 0

    def _sync(self):
        pass

    def _record(self):
        return _Event()

    def _check(self):
        pass

    def _admit(self, req, now):
        req.compiled = type("C", (), {"groups": 1})()
        req.admitted_s = now
        req.seen = 0
        self.requests.append(req)

    def _launch(self, active):
        held = sum(r.mem for r in self.requests if r.compiled is not None)
        self.worst = max(self.worst, held)
        for r in active:
            r.seen += 1
        self.next_segment = (self.next_segment + 1) % len(self.bounds)

    def _copy_out(self, r):
        r.result = (torch.zeros(1, dtype=torch.int64), torch.zeros(1, dtype=torch.int64))
        return 16


def test_finishing_queries_count_against_the_budget_until_harvested():
    # 12 queries of 300..700 bytes under a 1000-byte budget, all queued at t=0: a query
    # that finishes in a launch keeps its memory until that launch has been harvested,
    # so the next admission must not count on it
    need = {i: 300 + 100 * (i % 5) for i in range(12)}
    srv = _HostServer(FakeStore(1 << 16, need), budget=1000, max_slots=4, segments=3)
    reqs, stats = srv.serve([{"id": i} for i in range(12)], np.zeros(12), realtime=False)
    assert stats.completed == 12 and all(r.result is not None for r in reqs)
    assert srv.worst <= 1000, srv.worst
    assert stats.peak_held_bytes <= 1000
    assert stats.d2h_bytes == 16 * 12
