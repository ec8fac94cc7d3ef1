"""The seeded input generator: published SplitMix64 outputs, permutation validity, ranges."""
import numpy as np
import pytest

import datagen


def test_splitmix64_published_sequence():
    # SplitMix64 started from state 0 (Steele, Lea & Flood 2014; Vigna's splitmix64.c):
    # the first four outputs are the widely published seeding vectors below.
    expected = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]
    states = np.array([(0x9E3779B97F4A7C15 * (k + 1)) % (1 << 64) for k in range(4)], np.uint64)
    got = [int(v) for v in datagen.mix64(states)]
    assert got == expected


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 17, 2556, 65536, 200_003])
def test_perm_is_permutation(n):
    p = datagen.perm_i32(12345, 7, n)
    assert p.dtype == np.int32
    assert np.array_equal(np.sort(p), np.arange(n, dtype=np.int32))


def test_perm_elementwise_matches_slices():
    full = datagen.perm_i32(3, 9, 100_000)
    part = datagen.perm_i32(3, 9, 100_000, start=12_345, count=777)
    assert np.array_equal(full[12_345:12_345 + 777], part)
    assert not np.array_equal(full, np.arange(100_000))


def test_uniform_ranges_and_counter_access():
    x = datagen.uniform_i32(1, 2, 200_000, -5, 7)
    assert x.min() == -5 and x.max() == 7
    counts = np.bincount(x + 5)
    assert counts.min() > 0.9 * 200_000 / 13 and counts.max() < 1.1 * 200_000 / 13
    idx = np.array([0, 5, 199_999])
    assert np.array_equal(datagen.uniform_i32_at(1, 2, idx, -5, 7), x[idx])
    full = datagen.uniform_i32(1, 2, 1000, 0, (1 << 31) - 1)
    assert full.min() >= 0
    f = datagen.uniform_f32(4, 5, 100_000)
    assert f.dtype == np.float32 and f.min() >= 0.0 and f.max() < 1.0
    # exact multiples of 2^-24
    assert np.all((f.astype(np.float64) * 2 ** 24) % 1 == 0)


def test_bits_cover_sign():
    b = datagen.bits_i32(8, 9, 100_000)
    assert (b < 0).mean() > 0.45 and (b < 0).mean() < 0.55


def test_q1_tables_shape():
    t = datagen.q1_tables(11, 10_000)
    f, d = t["fact"], t["dim"]
    assert f["fk"].min() >= 0 and f["fk"].max() <= 2555
    assert f["a"].min() >= 1 and f["a"].max() <= 50
    assert f["b"].min() >= 0 and f["b"].max() <= 10
    assert f["c"].min() >= 1 and f["c"].max() <= 100_000
    assert np.array_equal(np.sort(d["key"]), np.arange(2556))
    # 2556 = 7 * 365 + 1: year code 0 appears 366 times, the others 365 times
    assert list(np.bincount(d["yr"])) == [366] + [365] * 6


def test_select_threshold_edges():
    assert datagen.select_threshold(0.0) == -1
    assert datagen.select_threshold(1.0) == (1 << 31) - 1
    assert datagen.select_threshold(0.5) == (1 << 30) - 1


def test_query_stream_well_formed():
    for q in range(200):
        query = datagen.ss_query(5, q)
        assert 1 <= len(query["joins"]) <= 4
        assert len({j["dim"] for j in query["joins"]}) == len(query["joins"])
        assert datagen.ss_group_count(query) <= datagen.SS_GROUP_LIMIT
        for j in query["joins"]:
            attrs = datagen.SS_DIMS[j["dim"]]["attrs"]
            for a, lo, hi in j["filters"]:
                assert 0 <= lo <= hi < attrs[a]
    arr = datagen.ss_arrivals(5, 1000, 100.0)
    assert np.all(np.diff(arr) >= 0) and 5.0 < arr[-1] < 15.0
