"""GPU parity of the single operators against the oracle (selection, projection, hash
join, radix sort), through the C ABI, at sizes spanning several tiles with ragged tails,
for every compiled tile shape, plus the empty and degenerate cases."""
import numpy as np
import pytest

import datagen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

I32_MIN, I32_MAX = -(1 << 31), (1 << 31) - 1
SIZES = [0, 1, 3, 4, 5, 127, 512, 4095, 4096, 4097, 65_537, 1_000_003]


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


# ------------------------------------------------------------------ selection

@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("variant", range(4))
def test_select_parity(crys, orc, n, variant):
    crys.crys_set_tile(crys.OP_SELECT, variant)
    x = datagen.uniform_i32(11 + n, datagen.STREAMS["sel.x"], n, 0, I32_MAX)
    xd = _dev(x)
    for sigma in (0.0, 0.1, 0.5, 1.0):
        hi = datagen.select_threshold(sigma)
        ref = orc.select(x, I32_MIN, hi)
        got = crys.select(xd, I32_MIN, hi, order_preserving=True).cpu().numpy()
        assert np.array_equal(got, ref), sigma                  # bit-exact, input order
        got = crys.select(xd, I32_MIN, hi, order_preserving=False).cpu().numpy()
        assert np.array_equal(np.sort(got), np.sort(ref)), sigma  # same multiset
    crys.crys_set_tile(crys.OP_SELECT, 0)


def test_select_ranges_and_negatives(crys, orc):
    x = datagen.uniform_i32(5, 9, 300_001, -1000, 1000)
    xd = _dev(x)
    for lo, hi in [(-5, 5), (1000, 1000), (-1000, -1000), (I32_MIN, I32_MAX), (3, 2), (2000, 3000)]:
        ref = orc.select(x, lo, hi)
        assert np.array_equal(crys.select(xd, lo, hi, True).cpu().numpy(), ref)
        assert np.array_equal(np.sort(crys.select(xd, lo, hi).cpu().numpy()), np.sort(ref))


def test_select_atomic_mode_keeps_order_inside_tiles(crys):
    # x = 0..n-1 in order: every tile's run must be increasing and runs are whole tiles
    n = 1 << 20
    xd = torch.arange(n, dtype=torch.int32, device="cuda")
    got = crys.select(xd, 0, I32_MAX).cpu().numpy()
    assert got.size == n and np.array_equal(np.sort(got), np.arange(n))
    breaks = np.flatnonzero(np.diff(got) != 1)
    assert breaks.size < n // 1024


# ------------------------------------------------------------------ projection

def _rel_err(got, ref):
    ref = ref.astype(np.float64)
    return np.abs(got.astype(np.float64) - ref) / np.maximum(np.abs(ref), 1e-30)


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("variant", range(4))
def test_project_parity(crys, orc, n, variant):
    crys.crys_set_tile(crys.OP_PROJECT, variant)
    x1 = datagen.uniform_f32(3 + n, datagen.STREAMS["proj.x1"], n)
    x2 = datagen.uniform_f32(3 + n, datagen.STREAMS["proj.x2"], n)
    d1, d2 = _dev(x1), _dev(x2)
    for op in (crys.PROJ_LINEAR, crys.PROJ_SIGMOID):
        got = crys.project(d1, d2, 2.0, 3.0, op).cpu().numpy()
        ref = orc.project(x1, x2, 2.0, 3.0, op)
        if n:
            assert _rel_err(got, ref).max() <= 1e-6
        # y = 0 and sigmoid(0) = 0.5 exactly
    z = torch.zeros(8, dtype=torch.float32, device="cuda")
    assert crys.project(z, z, 2.0, 3.0, crys.PROJ_SIGMOID).cpu().tolist() == [0.5] * 8
    crys.crys_set_tile(crys.OP_PROJECT, 0)


def test_project_in_place_and_negative_coefficients(crys, orc):
    n = 100_001
    x1 = datagen.uniform_f32(4, 1, n)
    x2 = datagen.uniform_f32(4, 2, n)
    d1, d2 = _dev(x1), _dev(x2)
    ref = orc.project(x1, x2, -2.5, 0.75, 1)
    crys.project(d1, d2, -2.5, 0.75, crys.PROJ_SIGMOID, out=d1)
    assert _rel_err(d1.cpu().numpy(), ref).max() <= 1e-6


# ------------------------------------------------------------------ hash join

@pytest.mark.parametrize("nb,np_", [(1, 1), (2, 1000), (1000, 4097), (1 << 16, 1_000_003), (3_000_017, 2_000_003)])
@pytest.mark.parametrize("variant", range(4))
def test_probe_parity(crys, orc, nb, np_, variant):
    crys.crys_set_tile(crys.OP_PROBE, variant)
    bk = datagen.perm_i32(21, datagen.STREAMS["join.bkey"], nb)
    bv = datagen.uniform_i32(21, datagen.STREAMS["join.bval"], nb, 1, 100)
    fk = datagen.uniform_i32(21, datagen.STREAMS["join.fk"], np_, 0, nb + nb // 3)  # ~25% misses
    pay = datagen.uniform_i32(21, datagen.STREAMS["join.pay"], np_, 1, 100)
    ht = crys.HashTable.build(_dev(bk), _dev(bv))
    s, m = crys.probe_aggregate(_dev(fk), _dev(pay), ht)
    assert (int(s.item()), int(m.item())) == orc.join_sum(bk, bv, fk, pay)
    crys.crys_set_tile(crys.OP_PROBE, 0)


@pytest.mark.parametrize("dense", [True, False])
def test_probe_identity_hash(crys, orc, dense):
    # identity hashing: collision-free for dense keys (capacity >= n), linear probing
    # resolves the collisions of sparse keys
    nb = 100_000
    bk = datagen.perm_i32(5, 1, nb) if dense else datagen.perm_i32(5, 1, nb) * 3 + 5  # never -1
    bv = datagen.uniform_i32(5, 2, nb, -100, 100)
    fk = datagen.uniform_i32(5, 3, 1_000_003, -10, 3 * nb)
    pay = datagen.uniform_i32(5, 4, 1_000_003, 1, 100)
    cap = crys.capacity_for(nb, crys.HASH_IDENT) * (1 if dense else 2)
    ht = crys.HashTable.build(_dev(bk), _dev(bv), capacity=cap, kind=crys.HASH_IDENT)
    s, m = crys.probe_aggregate(_dev(fk), _dev(pay), ht)
    assert (int(s.item()), int(m.item())) == orc.join_sum(bk, bv, fk, pay)


@pytest.mark.parametrize("nb", [1, 5000, 100_003])
def test_probe_direct_table(crys, orc, nb):
    # direct table: slot k holds key k (capacity = nb, no power of two); probe keys
    # outside [0, nb), negative ones included, are absent without a lookup
    bk = datagen.perm_i32(6, 1, nb)
    bv = datagen.uniform_i32(6, 2, nb, -100, 100)
    fk = datagen.uniform_i32(6, 3, 700_001, -50, nb + 50)
    pay = datagen.uniform_i32(6, 4, 700_001, 1, 100)
    ht = crys.HashTable.build(_dev(bk), _dev(bv), kind=crys.HASH_DIRECT)
    assert ht.capacity == nb
    s, m = crys.probe_aggregate(_dev(fk), _dev(pay), ht)
    assert (int(s.item()), int(m.item())) == orc.join_sum(bk, bv, fk, pay)
    slots = ht.slots.cpu().numpy().view(np.uint64)
    assert np.array_equal((slots & np.uint64(0xFFFFFFFF)).astype(np.int64), np.arange(nb))


def test_direct_table_rejects_keys_outside(crys):
    keys = np.array([0, 1, 2, 7], np.int32)              # 7 >= capacity 4
    ht = crys.HashTable(4, "cuda", kind=crys.HASH_DIRECT)
    crys.crys_hash_init(ht.struct)
    crys.crys_hash_build(_dev(keys), None, 4, [], ht.struct)
    assert crys.crys_device_errors(clear=True) & crys.DEV_BAD_KEY
    dup = np.array([0, 1, 1], np.int32)
    ht = crys.HashTable(4, "cuda", kind=crys.HASH_DIRECT)
    crys.crys_hash_init(ht.struct)
    crys.crys_hash_build(_dev(dup), None, 3, [], ht.struct)
    assert crys.crys_device_errors(clear=True) & crys.DEV_DUP_KEY


def test_hash_table_contents(crys):
    n = 50_000
    keys = datagen.perm_i32(3, 4, n) * 7 - 100_000       # sparse, negative keys
    vals = datagen.uniform_i32(3, 5, n, -50, 50)
    ht = crys.HashTable.build(_dev(keys), _dev(vals))
    slots = ht.slots.cpu().numpy().view(np.uint64)
    full = slots != np.uint64(0xFFFFFFFFFFFFFFFF)
    assert int(full.sum()) == n                          # exactly n occupied slots
    k = (slots[full] & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.int32)
    v = (slots[full] >> np.uint64(32)).astype(np.uint32).view(np.int32)
    order = np.argsort(k)
    ref = np.argsort(keys)
    assert np.array_equal(k[order], keys[ref]) and np.array_equal(v[order], vals[ref])


def _documented_home(keys, capacity):
    """Home slots as include/crystal.h states them for CRYS_HASH_MULT (numpy, wrapping)."""
    lg = capacity.bit_length() - 1
    k = keys.astype(np.int64).astype(np.uint64) & np.uint64(0xFFFFFFFF)
    if capacity <= 4096:
        return ((k * np.uint64(2654435769)) & np.uint64(0xFFFFFFFF)) >> np.uint64(32 - lg)
    return (k * np.uint64(0x9E3779B97F4A7C15)) >> np.uint64(64 - lg)


@pytest.mark.parametrize("n", [1000, 2048, 3000, 1 << 16, 1 << 22])
def test_hash_layout_follows_documented_home_slots(crys, n):
    """Every key of a linear-probing table sits at its documented home slot or after it
    with no empty slot in between (the layout callers may rely on, since they own the
    slots); dense keys 0..n-1 barely leave home under the multiplicative hash at every
    size (the 32-bit constant alone clustered them at 2^22: 1.3 extra slots per key)."""
    keys = datagen.perm_i32(5, 9, n)
    ht = crys.HashTable.build(_dev(keys), _dev(keys))
    cap = ht.capacity
    slots = ht.slots.cpu().numpy().view(np.uint64)
    full = slots != np.uint64(0xFFFFFFFFFFFFFFFF)
    pos = np.nonzero(full)[0]
    k = (slots[pos] & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.int32)
    home = _documented_home(k, cap).astype(np.int64)
    disp = (pos - home) % cap                      # slots walked past home (with wrap-around)
    # no empty slot between home and the key's slot: the run of occupied slots before
    # each key's slot is at least its displacement long
    empty = np.nonzero(~full)[0]
    run = np.empty(cap, np.int64)                  # occupied slots ending at each slot
    idx = np.arange(cap)
    last_empty = np.maximum.accumulate(np.where(~full, idx, -1))
    if empty.size:                                 # wrap-around: runs crossing slot 0
        last_empty = np.where(last_empty < 0, empty[-1] - cap, last_empty)
    run = idx - last_empty - 1
    assert np.all(disp <= run[pos])
    assert disp.mean() < 0.05


def test_filtered_build_and_payload_wrap(crys, orc):
    n = 20_000
    keys = datagen.perm_i32(8, 1, n)
    vals = np.full(n, I32_MAX, np.int32)
    attr = datagen.uniform_i32(8, 2, n, 0, 9)
    ht = crys.HashTable.build(_dev(keys), _dev(vals), filters=[(_dev(attr), 2, 4)])
    fk = datagen.uniform_i32(8, 3, 300_000, 0, n - 1)
    pay = np.full(300_000, I32_MAX, np.int32)
    s, m = crys.probe_aggregate(_dev(fk), _dev(pay), ht)
    keep = (attr >= 2) & (attr <= 4)
    assert (int(s.item()), int(m.item())) == orc.join_sum(keys[keep], vals[keep], fk, pay)


def test_probe_empty(crys):
    ht = crys.HashTable.build(torch.arange(4, dtype=torch.int32, device="cuda"))
    e = torch.empty(0, dtype=torch.int32, device="cuda")
    s, m = crys.probe_aggregate(e, e, ht)
    assert int(s.item()) == 0 and int(m.item()) == 0


# ------------------------------------------------------------------ sort

SORT_SIZES = [0, 1, 2, 31, 255, 256, 4095, 4096, 4097, 8191, 8193, 100_003, 1_048_579]


@pytest.mark.parametrize("n", SORT_SIZES)
@pytest.mark.parametrize("variant", range(4))
def test_sort_parity(crys, orc, n, variant):
    crys.crys_set_tile(crys.OP_SORT, variant)
    keys = datagen.bits_i32(17 + n, datagen.STREAMS["sort.key"], n)
    vals = np.arange(n, dtype=np.int32)
    ko, vo = crys.sort(_dev(keys), _dev(vals))
    rk, rv = orc.sort(keys, vals)
    assert np.array_equal(ko.cpu().numpy(), rk) and np.array_equal(vo.cpu().numpy(), rv)
    crys.crys_set_tile(crys.OP_SORT, 0)


@pytest.mark.parametrize("kind", ["equal", "sorted", "reversed", "extremes", "few", "bytes"])
def test_sort_adversarial(crys, orc, kind):
    n = 300_007
    rng = np.random.default_rng(5)
    if kind == "equal":
        keys = np.full(n, -7, np.int32)
    elif kind == "sorted":
        keys = np.arange(n, dtype=np.int32) - n // 2
    elif kind == "reversed":
        keys = (np.arange(n, dtype=np.int32) - n // 2)[::-1].copy()
    elif kind == "extremes":
        keys = rng.choice(np.array([I32_MIN, I32_MAX, 0, -1, 1], np.int32), size=n)
    elif kind == "few":
        keys = rng.integers(-3, 3, size=n).astype(np.int32)
    else:  # a single non-zero byte per key: passes that see only one digit
        keys = (rng.integers(0, 256, size=n) << 16).astype(np.int32)
    vals = rng.integers(I32_MIN, I32_MAX, size=n, dtype=np.int64).astype(np.int32)
    ko, vo = crys.sort(_dev(keys), _dev(vals))
    rk, rv = orc.sort(keys, vals)
    assert np.array_equal(ko.cpu().numpy(), rk) and np.array_equal(vo.cpu().numpy(), rv)


# ------------------------------------------------------------------ input generator

def test_device_generator_matches_host(crys):
    import datagen.device as dgd
    for n in (0, 1, 1000, 123_457):
        assert np.array_equal(dgd.uniform_i32(3, 9, n, -7, 1_000_000).cpu().numpy(),
                              datagen.uniform_i32(3, 9, n, -7, 1_000_000))
        assert np.array_equal(dgd.uniform_f32(3, 9, n).cpu().numpy(), datagen.uniform_f32(3, 9, n))
        assert np.array_equal(dgd.bits_i32(3, 9, n).cpu().numpy(), datagen.bits_i32(3, 9, n))
        assert np.array_equal(dgd.perm_i32(3, 9, max(n, 1)).cpu().numpy(), datagen.perm_i32(3, 9, max(n, 1)))
    big = dgd.uniform_i32(4, 5, 1 << 24, 0, I32_MAX).cpu().numpy()
    idx = np.array([0, 1, 12345, (1 << 24) - 1])
    assert np.array_equal(big[idx], datagen.uniform_i32_at(4, 5, idx, 0, I32_MAX))


@pytest.mark.parametrize("n", [0, 1, 5, 4097, 1_000_003, 1 << 22])
@pytest.mark.parametrize("sigma", [0.0, 0.3, 1.0])
def test_select_strawman_parity(crys, orc, n, sigma):
    # the independent-threads selection: input order, like the order-preserving mode
    x = datagen.uniform_i32(17 + n, datagen.STREAMS["sel.x"], n, 0, I32_MAX)
    hi = datagen.select_threshold(sigma)
    xd = _dev(x)
    out = torch.empty(max(1, n), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    tb = crys.crys_select_strawman(None, n, I32_MIN, hi, None, None, None, -1)
    temp = crys.scratch(tb, "cuda")
    crys.crys_select_strawman(xd, n, I32_MIN, hi, out, cnt, temp, tb)
    ref = orc.select(x, I32_MIN, hi)
    c = int(cnt.item())
    assert c == ref.size and np.array_equal(out[:c].cpu().numpy(), ref)
