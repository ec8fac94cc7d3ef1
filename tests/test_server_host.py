"""Host-side logic of the serving loop (no GPU): admission by slots and memory, requests
that can never fit, segment bounds of the circular scan."""
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
