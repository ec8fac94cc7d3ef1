"""GPU parity of the operators built on unstable radix partitioning, through the C ABI:
the MSB radix sort (Section 4.4, the paper's GPU sort) and the radix-partitioned hash
join (Section 4.3), against the oracle.

The MSB sort is unstable, so its parity is: the key sequence equals the oracle's
(a stable sort's key sequence is the unique sorted order), and the (key, value) pairs are
the input pairs (compared as a multiset in (key, value) order).  The join is exact: the
int64 sum and the match count equal the oracle's."""
import numpy as np
import pytest

import datagen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

I32_MIN, I32_MAX = -(1 << 31), (1 << 31) - 1


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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _check_unstable_sort(crys, orc, keys, vals):
    ko, vo = crys.sort_msb(_dev(keys), _dev(vals))
    ko, vo = ko.cpu().numpy(), vo.cpu().numpy()
    rk, rv = orc.sort(keys, vals)
    assert np.array_equal(ko, rk)                              # exact key order
    got = np.lexsort((vo, ko))
    ref = np.lexsort((rv, rk))
    assert np.array_equal(ko[got], rk[ref]) and np.array_equal(vo[got], rv[ref])   # same pairs


MSB_SIZES = [0, 1, 2, 31, 255, 256, 4095, 4096, 4097, 8191, 8193, 100_003, 1_048_579, 5_000_011]


@pytest.mark.parametrize("n", MSB_SIZES)
def test_msb_sort_parity(crys, orc, n):
    keys = datagen.bits_i32(23 + n, datagen.STREAMS["sort.key"], n)
    _check_unstable_sort(crys, orc, keys, np.arange(n, dtype=np.int32))


@pytest.mark.parametrize("kind", ["equal", "sorted", "reversed", "extremes", "few", "bytes", "top16", "low16"])
def test_msb_sort_adversarial(crys, orc, kind):
    n = 300_007
    rng = np.random.default_rng(9)
    if kind == "equal":          # one bucket of every row: the large-bucket path
        keys = np.full(n, -7, np.int32)
    elif kind == "sorted":
        keys = np.arange(n, dtype=np.int32) - n // 2
    elif kind == "reversed":
        keys = (np.arange(n, dtype=np.int32) - n // 2)[::-1].copy()
    elif kind == "extremes":
        keys = rng.choice(np.array([I32_MIN, I32_MAX, 0, -1, 1], np.int32), size=n)
    elif kind == "few":
        keys = rng.integers(-3, 3, size=n).astype(np.int32)
    elif kind == "bytes":
        keys = (rng.integers(0, 256, size=n) << 16).astype(np.int32)
    elif kind == "top16":        # equal top 16 bits, random low bits: one bucket, many chunks
        keys = ((0x1234 << 16) | rng.integers(0, 1 << 16, size=n)).astype(np.int32)
    else:                        # random top bits, few low-bit values
        keys = ((rng.integers(-(1 << 15), 1 << 15, size=n) << 16) | rng.integers(0, 4, size=n)).astype(np.int32)
    vals = rng.integers(I32_MIN, I32_MAX, size=n, dtype=np.int64).astype(np.int32)
    _check_unstable_sort(crys, orc, keys, vals)


def test_msb_sort_scratch_and_overlap(crys):
    L = crys.lib()
    import ctypes as C
    size = C.c_size_t(0)
    assert L.crys_sort_msb(None, None, None, None, 1 << 20, None, C.byref(size), None) == crys.OK
    assert size.value >= 8 * (1 << 20)
    k = torch.zeros(1024, dtype=torch.int32, device="cuda")
    t = torch.empty(size.value, dtype=torch.uint8, device="cuda")
    # output aliasing the input is refused
    assert crys.lib().crys_sort_msb(C.c_void_p(k.data_ptr()), C.c_void_p(k.data_ptr()), C.c_void_p(k.data_ptr()),
                                    C.c_void_p(k.data_ptr()), 1024, C.c_void_p(t.data_ptr()), C.byref(size),
                                    None) == crys.EINVAL


# ------------------------------------------------------------------ partitioned join

def _join(crys, bk, bv, fk, pay):
    s, m = crys.join_partitioned(_dev(bk), _dev(bv), _dev(fk), _dev(pay))
    return int(s.item()), int(m.item())


@pytest.mark.parametrize("nb", [1, 100, 2048, 2049, 4096, 5000, 70_001, 1 << 20])
def test_partitioned_join_parity(crys, orc, nb):
    # every partitioning depth: none (<= 2048 build rows), one pass, two passes; probe
    # keys outside the build keys (negative ones included) miss
    bk = datagen.perm_i32(31, 1, nb)
    bv = datagen.uniform_i32(31, 2, nb, -100, 100)
    npr = 1_000_003
    fk = datagen.uniform_i32(31, 3, npr, -50, nb + nb // 3)
    pay = datagen.uniform_i32(31, 4, npr, 1, 100)
    assert _join(crys, bk, bv, fk, pay) == orc.join_sum(bk, bv, fk, pay)


def test_partitioned_join_skewed_partition(crys, orc):
    # build keys whose hash top bits are all equal: one partition holds every build row,
    # too large for shared memory, so its table is built in scratch
    cand = np.arange(0, 1 << 26, dtype=np.int64)
    top = ((cand * 2654435769) & 0xFFFFFFFF) >> 28
    bk = cand[top == 5][:20_000].astype(np.int32)
    assert bk.size == 20_000
    bv = datagen.uniform_i32(32, 2, bk.size, 1, 100)
    fk = np.concatenate([bk, datagen.uniform_i32(32, 3, 200_000, 0, 1 << 26)]).astype(np.int32)
    pay = datagen.uniform_i32(32, 4, fk.size, 1, 100)
    assert _join(crys, bk, bv, fk, pay) == orc.join_sum(bk, bv, fk, pay)


def test_partitioned_join_wrap_and_empty(crys, orc):
    n = 30_000
    bk = datagen.perm_i32(33, 1, n) * 3 - 40_000          # sparse, negative keys
    bv = np.full(n, I32_MAX, np.int32)
    fk = datagen.uniform_i32(33, 3, 400_000, -40_000, 50_000)
    pay = np.full(400_000, I32_MAX, np.int32)
    assert _join(crys, bk, bv, fk, pay) == orc.join_sum(bk, bv, fk, pay)
    e = np.empty(0, np.int32)
    assert _join(crys, e, e, fk, pay) == (0, 0)
    assert _join(crys, bk, bv, e, e) == (0, 0)


def test_partitioned_join_matches_direct_probe(crys):
    nb = 1 << 18
    bk = datagen.perm_i32(34, 1, nb)
    bv = datagen.uniform_i32(34, 2, nb, 1, 100)
    fk = _dev(datagen.uniform_i32(34, 3, 3_000_000, 0, nb - 1))
    pay = _dev(datagen.uniform_i32(34, 4, 3_000_000, 1, 100))
    ht = crys.HashTable.build(_dev(bk), _dev(bv))
    s1, m1 = crys.probe_aggregate(fk, pay, ht)
    s2, m2 = crys.join_partitioned(_dev(bk), _dev(bv), fk, pay)
    assert int(s1.item()) == int(s2.item()) and int(m1.item()) == int(m2.item()) == 3_000_000
