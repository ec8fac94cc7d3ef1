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
