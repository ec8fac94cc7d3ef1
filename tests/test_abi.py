"""The C-ABI library loads and exports every symbol include/crystal.h declares; host-side
argument checks answer without touching a GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def crys():
    from paper_2003_01178_gb300 import _build
    _build.build()
    import paper_2003_01178_gb300 as crys
    crys.lib()
    return crys


def _declared():
    text = open(os.path.join(ROOT, "include", "crystal.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(crys_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(crys):
    names = _declared()
    assert len(names) >= 15
    L = crys.lib()
    for n in names:
        assert hasattr(L, n), n


def test_strerror_and_tiles(crys):
    assert crys.strerror(crys.OK) == "ok"
    assert "argument" in crys.strerror(crys.EINVAL)
    for op in range(crys.NUM_OPS):
        v = crys.crys_tile_variants(op)
        assert 1 <= len(v) <= 4 and all(t % 32 == 0 and i > 0 for t, i in v)
    assert crys.crys_tile_variants(0)[3] == (128, 4)      # the paper's tile shape is available
    # the tagged scan has shapes of its own; its default runs one 1024-thread block per SM
    # (the smallest table's entries in shared memory), another two 512-thread blocks; a
    # list entry holds a 3-bit item slot, so at most 8 items per thread
    tagged = crys.crys_tile_variants(crys.OP_TAGGED_SCAN)
    assert crys.NUM_OPS == 7 and tagged[0] == (1024, 4) and (512, 4) in tagged
    assert all(i <= 8 and t <= 1024 for t, i in tagged)
    with pytest.raises(crys.CrystalError):
        crys.crys_set_tile(0, 99)
    crys.crys_set_tile(0, 1)
    assert crys.crys_get_tile(0) == 1
    crys.crys_set_tile(0, 0)


def test_host_side_validation_without_gpu(crys):
    L = crys.lib()
    size = C.c_size_t(0)
    # size queries
    assert L.crys_select(None, 1000, 0, 1, None, None, 1, None, C.byref(size), None) == crys.OK
    assert size.value >= 8
    assert L.crys_select(None, 1000, 0, 1, None, None, 0, None, C.byref(size), None) == crys.OK
    assert size.value == 0
    assert L.crys_sort(None, None, None, None, 1 << 20, None, C.byref(size), None) == crys.OK
    assert size.value >= 8 * (1 << 20)
    # rejected before any launch
    assert L.crys_select(None, -1, 0, 1, None, None, 0, None, None, None) == crys.EINVAL
    assert L.crys_select(None, 10, 0, 1, None, None, 2, None, None, None) == crys.EINVAL
    assert L.crys_project(None, None, 10, 1.0, 1.0, 5, None, None) == crys.EINVAL
    assert L.crys_project(C.c_void_p(16), C.c_void_p(16), 10, 1.0, 1.0, 0, C.c_void_p(20), None) == crys.EINVAL
    bad = crys.crys_hash(C.c_void_p(4096), 3)
    assert L.crys_hash_init(C.byref(bad), None) == crys.EINVAL
    assert L.crys_sort(None, None, None, None, 1 << 31, None, None, None) == crys.EINVAL
    ok = crys.crys_hash(C.c_void_p(4096), 8)
    assert L.crys_hash_build(C.c_void_p(4096), None, 100, None, 0, C.byref(ok), None) == crys.EFULL
    plan = crys.crys_plan()
    plan.n_joins = 2
    plan.joins[0].group_card = 100
    plan.joins[1].group_card = 7
    g = C.c_int64(0)
    assert L.crys_plan_groups(C.byref(plan), C.byref(g)) == crys.OK and g.value == 700
    plan.joins[1].group_card = -1
    assert L.crys_plan_groups(C.byref(plan), C.byref(g)) == crys.EINVAL
    t = crys.crys_table()
    t.n_cols = 0
    assert L.crys_run_plan(C.byref(t), C.byref(plan), None) == crys.EINVAL
    assert L.crys_run_plans(C.byref(t), None, 40, 0, 0, 0, None) == crys.EINVAL


def test_generator_library_exports(crys):
    import datagen.device as dgd
    L = dgd.lib()
    for n in ("dg_uniform_i32", "dg_uniform_f32", "dg_bits_i32", "dg_perm_i32"):
        assert hasattr(L, n)


def test_product_does_not_import_oracle():
    """The package imports neither the oracle nor the input generator (it owns no workload)."""
    import subprocess
    import sys
    code = ("import sys; sys.path.insert(0, %r); import paper_2003_01178_gb300, "
            "paper_2003_01178_gb300.starschema, paper_2003_01178_gb300.server; "
            "assert 'oracle' not in sys.modules, 'oracle imported'; "
            "assert 'datagen' not in sys.modules, 'the input generator imported'" % ROOT)
    subprocess.check_call([sys.executable, "-c", code])


def test_tagged_scan_scratch_sizing(crys):
    """Host-side sizing of the query bitmaps (no device access): one entry of 8 bytes per
    slot of each distinct (fact column, direct table) pair, 16-byte rounded; 0 when a
    join is on a table of another kind."""
    L = crys.lib()
    t = crys.crys_table()
    t.n_cols = 3
    t.n_rows = 1000
    for c in range(3):
        t.cols[c] = 4096 * (c + 1)

    def plan(fk, slots, cap, kind):
        p = crys.crys_plan()
        p.n_joins = 1
        p.joins[0].fk_col = fk
        p.joins[0].ht = crys.crys_hash(C.c_void_p(slots), cap, kind)
        p.agg_a = 2
        p.d_sums = 1 << 20
        return p

    D = crys.HASH_DIRECT
    plans = [plan(0, 1 << 16, 1001, D), plan(0, 1 << 16, 1001, D), plan(1, 1 << 24, 7, D)]
    arr = (crys.crys_plan * 3)(*plans)
    b = C.c_int64(-1)
    assert L.crys_run_plans_tagged_bytes(C.byref(t), arr, 3, C.byref(b)) == crys.OK
    assert b.value == (1001 * 8 + 15) // 16 * 16 + (7 * 8 + 15) // 16 * 16
    plans[2] = plan(1, 1 << 24, 8, crys.HASH_MULT)
    arr = (crys.crys_plan * 3)(*plans)
    assert L.crys_run_plans_tagged_bytes(C.byref(t), arr, 3, C.byref(b)) == crys.OK and b.value == 0
    # a power-of-two capacity is required of the probing kinds, not of direct tables
    plans[2] = plan(1, 1 << 24, 7, crys.HASH_MULT)
    arr = (crys.crys_plan * 3)(*plans)
    assert L.crys_run_plans_tagged_bytes(C.byref(t), arr, 3, C.byref(b)) == crys.EINVAL
    assert L.crys_run_plans_tagged_bytes(C.byref(t), arr, 40, C.byref(b)) == crys.EINVAL
    assert L.crys_run_plans_tagged_bytes(C.byref(t), arr, 1, None) == crys.EINVAL
    # misaligned scratch is rejected before anything is enqueued
    assert L.crys_run_plans_tagged(C.byref(t), arr, 1, 0, 1000, 0, C.c_void_p(8), 64, None) == crys.EINVAL
    assert L.crys_run_plans_tagged(C.byref(t), arr, 1, 2, 1000, 0, None, 0, None) == crys.EINVAL


def test_replayable_launch_host_checks(crys):
    """Argument-block entry points: size query, and rejection of bad arguments before
    any device work (no GPU needed)."""
    L = crys.lib()
    b = C.c_int64(0)
    assert L.crys_tagged_block_bytes(C.byref(b)) == crys.OK and b.value > 0 and b.value % 256 == 0
    assert L.crys_tagged_block_bytes(None) == crys.EINVAL
    t = crys.crys_table()
    t.n_cols = 1
    t.n_rows = 100
    t.cols[0] = 4096
    p = crys.crys_plan()
    p.d_sums = 1 << 20
    arr = (crys.crys_plan * 1)(p)
    hb = (C.c_uint8 * b.value)()
    z = (C.c_int32 * 1)(0)
    args = dict(fact=C.byref(t), plans=arr)
    # no block, no plans, bad flags, bad zero list, misaligned scratch, odd row start
    assert L.crys_tagged_prepare(C.byref(t), arr, 1, 0, 100, 0, z, 0, C.c_void_p(4096), 64, None) == crys.EINVAL
    assert L.crys_tagged_prepare(C.byref(t), arr, 0, 0, 100, 0, z, 0, C.c_void_p(4096), 64, hb) == crys.EINVAL
    assert L.crys_tagged_prepare(C.byref(t), arr, 1, 0, 100, 0x10, z, 0, C.c_void_p(4096), 64, hb) == crys.EINVAL
    assert L.crys_tagged_prepare(C.byref(t), arr, 1, 0, 100, 0, None, 1, C.c_void_p(4096), 64, hb) == crys.EINVAL
    assert L.crys_tagged_prepare(C.byref(t), arr, 1, 0, 100, 0, z, 0, C.c_void_p(4100), 64, hb) == crys.EINVAL
    assert L.crys_tagged_prepare(C.byref(t), arr, 1, 2, 100, 0, z, 0, C.c_void_p(4096), 64, hb) == crys.EINVAL
    assert L.crys_tagged_launch(None, None) == crys.EINVAL
    del args


def test_debug_stall_arguments(crys):
    """The wait-bound test hook validates its arguments on the host."""
    L = crys.lib()
    assert L.crys_debug_stall(crys.OP_PROJECT, 1, 1_000_000) == crys.EINVAL
    assert L.crys_debug_stall(crys.OP_SELECT, -1, 1_000_000) == crys.EINVAL
    assert L.crys_debug_stall(crys.OP_SELECT, 1, 10) == crys.EINVAL
    assert L.crys_debug_stall(crys.OP_SORT, 1, 3_000_000_000) == crys.EINVAL


def test_tuner_persists_tile_shapes(crys, tmp_path, monkeypatch):
    """The autotuner stores each operator's choice as a tile shape: loading finds that
    shape's variant even if the variant list was reordered, and ignores a shape that is
    no longer compiled or an entry in another form (no GPU needed: choices are host state)."""
    import json
    from paper_2003_01178_gb300 import tuner
    monkeypatch.setattr(tuner, "_key", lambda: "test-device")
    path = str(tmp_path / "tiles.json")
    op = crys.OP_TAGGED_SCAN
    variants = crys.crys_tile_variants(op)
    try:
        crys.crys_set_tile(op, 2)
        tuner.save(path)
        stored = json.load(open(path))["test-device"]
        assert stored[crys.OP_NAMES[op]] == list(variants[2])
        crys.crys_set_tile(op, 0)
        assert tuner.load(path) and crys.crys_get_tile(op) == 2
        stored[crys.OP_NAMES[op]] = [96, 3]                 # not a compiled shape
        stored[crys.OP_NAMES[crys.OP_SELECT]] = 1            # an index (another form)
        json.dump({"test-device": stored}, open(path, "w"))
        crys.crys_set_tile(op, 1)
        crys.crys_set_tile(crys.OP_SELECT, 3)
        assert tuner.load(path)
        assert crys.crys_get_tile(op) == 1 and crys.crys_get_tile(crys.OP_SELECT) == 3
    finally:
        for o in range(crys.NUM_OPS):
            crys.crys_set_tile(o, 0)
