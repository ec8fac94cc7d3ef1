"""Conditions only the GPU can see are reported through the sticky device error word,
without trapping or hanging: duplicate and reserved keys, a full table, group codes out
of range.  (All waits in the kernels are bounded; these cases do not wait at all.)"""
import numpy as np
import pytest

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
    crys.crys_device_errors(clear=True)


def test_duplicate_key_flag(crys):
    keys = torch.tensor([1, 2, 3, 2], dtype=torch.int32, device="cuda")
    crys.HashTable.build(keys)
    assert crys.crys_device_errors(clear=True) & crys.DEV_DUP_KEY


def test_reserved_key_flag(crys):
    keys = torch.tensor([5, -1, 7, 9], dtype=torch.int32, device="cuda")
    crys.HashTable.build(keys)
    assert crys.crys_device_errors(clear=True) & crys.DEV_BAD_KEY


def test_table_full_flag_without_hang(crys):
    keys = torch.arange(100, dtype=torch.int32, device="cuda")
    attr = torch.zeros(100, dtype=torch.int32, device="cuda")
    # a filter that keeps every row defeats the host-side capacity check
    ht = crys.HashTable(16, "cuda")
    crys.crys_hash_init(ht.struct)
    crys.crys_hash_build(keys, None, 100, [(attr, 0, 0)], ht.struct)
    assert crys.crys_device_errors(clear=True) & crys.DEV_TABLE_FULL
    # probing a full table still terminates (bounded by the capacity)
    s, m = crys.probe_aggregate(torch.arange(200, dtype=torch.int32, device="cuda"),
                                torch.ones(200, dtype=torch.int32, device="cuda"), ht)
    assert int(m.item()) == 16
    assert crys.crys_device_errors(clear=True) == 0


def test_bad_group_code_flag(crys):
    keys = torch.arange(10, dtype=torch.int32, device="cuda")
    codes = torch.tensor([0, 1, 2, 9, 0, 1, 2, 0, 1, 2], dtype=torch.int32, device="cuda")
    ht = crys.HashTable.build(keys, codes)
    fk = torch.arange(10, dtype=torch.int32, device="cuda").repeat(100)
    price = torch.ones(1000, dtype=torch.int32, device="cuda")
    sums, counts = crys.run_plan([fk, price], [], [(0, ht, 3)], ("sum", 1, None))
    assert crys.crys_device_errors(clear=True) & crys.DEV_BAD_GROUP
    assert counts.cpu().tolist() == [300, 300, 300]     # the row with code 9 is dropped


def test_host_rejections_enqueue_nothing(crys):
    before = crys.crys_launch_count()
    x = torch.zeros(16, dtype=torch.int32, device="cuda")
    with pytest.raises(crys.CrystalError):
        crys.crys_select(x[1:], 15, 0, 1, x, torch.zeros(1, dtype=torch.int64, device="cuda"), 0)
    with pytest.raises(crys.CrystalError):
        crys.crys_sort(x, x, x, x, 16, torch.empty(16, dtype=torch.uint8, device="cuda"), 16)
    assert crys.crys_launch_count() == before


def _flags(crys, clear=False):
    return crys.crys_device_errors(clear=clear)


def test_select_lookback_timeout_is_reported_and_stays_in_its_call(crys, orc):
    """A predecessor tile that never publishes (tile ids start at 5): the order-preserving
    selection's look-back gives up after its 2 ms bound, the call returns promptly with
    CRYS_DEV_TIMEOUT set, and a later call - with the error word NOT cleared - is exact."""
    import time
    import datagen
    crys.crys_device_errors(clear=True)
    x = torch.from_numpy(datagen.uniform_i32(9, datagen.STREAMS["sel.x"], 1 << 22, 0, (1 << 31) - 1)).cuda()
    hi = datagen.select_threshold(0.5)
    crys.crys_debug_stall(crys.OP_SELECT, 5, 2_000_000)
    t0 = time.perf_counter()
    got = crys.select(x, -(1 << 31), hi, order_preserving=True)   # synchronises on the count
    elapsed = time.perf_counter() - t0
    assert elapsed < 1.5, elapsed
    assert _flags(crys) & crys.DEV_TIMEOUT
    assert got.numel() < x.numel()                  # the call's output is incomplete
    # the next call carries no abort from the one that gave up
    got = crys.select(x, -(1 << 31), hi, order_preserving=True).cpu().numpy()
    assert np.array_equal(got, orc.select(x.cpu().numpy(), -(1 << 31), hi))
    assert _flags(crys, clear=True) == crys.DEV_TIMEOUT   # only the stalled call's bit
    assert _flags(crys) == 0


def test_sort_lookback_timeout_is_reported_and_stays_in_its_call(crys, orc):
    import time
    import datagen
    crys.crys_device_errors(clear=True)
    n = 300_001
    keys = torch.from_numpy(datagen.bits_i32(9, datagen.STREAMS["sort.key"], n)).cuda()
    vals = torch.arange(n, dtype=torch.int32, device="cuda")
    crys.crys_debug_stall(crys.OP_SORT, 3, 2_000_000)
    t0 = time.perf_counter()
    crys.sort(keys, vals)
    torch.cuda.synchronize()
    assert time.perf_counter() - t0 < 1.5
    assert _flags(crys) & crys.DEV_TIMEOUT
    ko, vo = crys.sort(keys, vals)
    rk, rv = orc.sort(keys.cpu().numpy(), vals.cpu().numpy())
    assert np.array_equal(ko.cpu().numpy(), rk) and np.array_equal(vo.cpu().numpy(), rv)
    assert _flags(crys, clear=True) == crys.DEV_TIMEOUT
    assert _flags(crys) == 0

