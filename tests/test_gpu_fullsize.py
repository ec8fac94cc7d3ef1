"""Parity at the benchmark's full sizes, with the bench's seeded inputs and the default
tile shapes: every workload the bench times, checked against the oracle element by
element where the oracle finishes in seconds (selection, the join sums, the fused query,
a served batch over a row prefix and two of its queries over all rows), on sampled
outputs (projection) or through properties that fix the result at any size (the stable
sort: ordered keys, row ids a permutation, each output pair an input pair, equal keys in
row-id order)."""
import numpy as np
import pytest

import datagen

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
torch = pytest.importorskip("torch")

SEED = 0xC0FFEE + 4   # the bench's default seed
I32_MIN, I32_MAX = -(1 << 31), (1 << 31) - 1


@pytest.fixture(scope="module")
def crys():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2003_01178_gb300 import _build
    _build.build()
    import paper_2003_01178_gb300 as crys
    crys.crys_device_errors(clear=True)
    for op in range(crys.NUM_OPS):
        crys.crys_set_tile(op, 0)
    yield crys
    assert crys.crys_device_errors(clear=True) == 0


@pytest.fixture(scope="module")
def threads(orc):
    return orc.hardware_threads()


def test_select_full_size(crys, orc, threads):
    import datagen.device as dgd
    n = 1 << 29
    x = dgd.uniform_i32(SEED, datagen.STREAMS["sel.x"], n, 0, I32_MAX)
    xh = x.cpu().numpy()
    for sigma in (0.0, 0.5, 1.0):
        hi = datagen.select_threshold(sigma)
        got = crys.select(x, I32_MIN, hi, order_preserving=True)
        ref = orc.select(xh, I32_MIN, hi, threads=threads)
        assert got.numel() == ref.size
        assert np.array_equal(got.cpu().numpy(), ref)
    # atomic (unordered) mode: the same multiset, compared element by element once both
    # sides are put in ascending order (torch's sort as the canonicalising step)
    hi = datagen.select_threshold(0.3)
    got = crys.select(x, I32_MIN, hi, order_preserving=False)
    ref = orc.select(xh, I32_MIN, hi, threads=threads)
    assert got.numel() == ref.size
    got_sorted = torch.sort(got).values.cpu().numpy()
    ref_sorted = torch.sort(torch.from_numpy(ref).cuda()).values.cpu().numpy()
    assert np.array_equal(got_sorted, ref_sorted)


def test_project_full_size_sampled(crys, orc):
    import datagen.device as dgd
    n = 1 << 29
    x1 = dgd.uniform_f32(SEED, datagen.STREAMS["proj.x1"], n)
    x2 = dgd.uniform_f32(SEED, datagen.STREAMS["proj.x2"], n)
    y = torch.empty_like(x1)
    sample = np.concatenate([np.random.default_rng(5).integers(0, n, 1 << 22), [0, n - 1]])
    idx = torch.from_numpy(sample).cuda()
    for op in (crys.PROJ_LINEAR, crys.PROJ_SIGMOID):
        crys.crys_project(x1, x2, n, 2.0, 3.0, op, y)
        got = y[idx].cpu().numpy()
        ref = orc.project(x1[idx].cpu().numpy(), x2[idx].cpu().numpy(), 2.0, 3.0, op)
        assert np.allclose(got, ref, rtol=1e-6, atol=0)


@pytest.mark.parametrize("lg", [10, 27])
def test_join_full_size(crys, orc, threads, lg):
    """The direct probe and the radix-partitioned join, both against the oracle."""
    import datagen.device as dgd
    nb, n = 1 << lg, 1 << 28
    bk = dgd.perm_i32(SEED, datagen.STREAMS["join.bkey"], nb)
    bv = dgd.uniform_i32(SEED, datagen.STREAMS["join.bval"], nb, 1, 100)
    fk = dgd.uniform_i32(SEED, datagen.STREAMS["join.fk"], n, 0, nb - 1)
    pay = dgd.uniform_i32(SEED, datagen.STREAMS["join.pay"], n, 1, 100)
    ht = crys.HashTable.build(bk, bv)
    s, m = crys.probe_aggregate(fk, pay, ht)
    ref = orc.join_sum(bk.cpu().numpy(), bv.cpu().numpy(), fk.cpu().numpy(), pay.cpu().numpy(), threads=threads)
    assert (int(s.item()), int(m.item())) == ref
    assert int(m.item()) == n                    # every foreign key names a build key
    del ht
    s, m = crys.join_partitioned(bk, bv, fk, pay)
    assert (int(s.item()), int(m.item())) == ref


def test_sort_full_size_properties(crys):
    import datagen.device as dgd
    n = 1 << 28
    keys = dgd.bits_i32(SEED, datagen.STREAMS["sort.key"], n)
    vals = torch.arange(n, dtype=torch.int32, device="cuda")
    ko, vo = crys.sort(keys, vals)
    k = ko.cpu().numpy().astype(np.int64)
    v = vo.cpu().numpy().astype(np.int64)
    kin = keys.cpu().numpy()
    dk = np.diff(k)
    assert np.all(dk >= 0)                                    # ordered (signed)
    assert np.all(np.diff(v)[dk == 0] > 0)                    # stable: equal keys by row id
    seen = np.zeros(n, np.uint8)
    seen[v] = 1
    assert seen.all()                                         # row ids a permutation
    assert np.array_equal(kin[v], k.astype(np.int32))         # each pair is an input pair


def test_msb_sort_full_size_properties(crys):
    """The unstable MSB sort at 2^28 keys: ordered keys, row ids a permutation, and each
    output pair an input pair (what fixes an unstable sort's result)."""
    import datagen.device as dgd
    n = 1 << 28
    keys = dgd.bits_i32(SEED, datagen.STREAMS["sort.key"], n)
    vals = torch.arange(n, dtype=torch.int32, device="cuda")
    ko, vo = crys.sort_msb(keys, vals)
    k = ko.cpu().numpy()
    v = vo.cpu().numpy().astype(np.int64)
    assert np.all(np.diff(k.astype(np.int64)) >= 0)
    seen = np.zeros(n, np.uint8)
    seen[v] = 1
    assert seen.all()
    assert np.array_equal(keys.cpu().numpy()[v], k)


def test_q1_full_size(crys, orc, threads):
    import datagen.device as dgd
    for n in (1 << 22, 1 << 28):
        t = dgd.q1_tables(SEED, n)
        f, d = t["fact"], t["dim"]
        ht = crys.HashTable.build(d["key"], d["yr"], filters=[(d["yr"], 3, 3)])
        sums, _ = crys.run_plan([f["fk"], f["a"], f["b"], f["c"]], [(1, I32_MIN, 24), (2, 1, 3)],
                                [(0, ht, 0)], ("mul", 3, 2))
        fh = {k: v.cpu().numpy() for k, v in f.items()}
        dh = {k: v.cpu().numpy() for k, v in d.items()}
        assert int(sums[0].item()) == orc.q1_run(fh, dh, threads=threads)


def test_served_batch_full_size(crys, orc, threads):
    """One batch of the bench (32 queries, 600M fact rows) in the tagged shared scan:
    every query over the first 16M rows, two queries over all rows."""
    import datagen.device as dgd
    from paper_2003_01178_gb300.starschema import ResidentStarSchema, Schema
    n = 600_000_000
    t = dgd.ss_tables(SEED, n)
    store = ResidentStarSchema(Schema.from_spec(datagen.SS_FACT_COLS, datagen.SS_DIMS), t["fact"], t["dims"])
    queries = [datagen.ss_query(SEED, i) for i in range(32)]       # batch 0 of the bench
    host = {"fact": {k: v.cpu().numpy() for k, v in t["fact"].items()},
            "dims": {d: {k: v.cpu().numpy() for k, v in cols.items()} for d, cols in t["dims"].items()}}
    prefix = 16_000_000
    cqs = [store.compile(q) for q in queries]
    store.run_shared(cqs, 0, prefix)
    for cq, q in zip(cqs, queries):
        rs, rc = orc.ss_run(host, q, threads=threads, fact_rows=prefix)
        assert np.array_equal(cq.sums.cpu().numpy(), rs) and np.array_equal(cq.counts.cpu().numpy(), rc)
    cqs = [store.compile(q) for q in queries]
    store.run_shared(cqs)
    for i in (0, 17):
        rs, rc = orc.ss_run(host, queries[i], threads=threads)
        assert np.array_equal(cqs[i].sums.cpu().numpy(), rs) and np.array_equal(cqs[i].counts.cpu().numpy(), rc)
    crys.check_device_errors()
