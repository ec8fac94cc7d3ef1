"""Python binding of libcrystal.so, the GB300 (sm_103a) tile-based query operators.

The functions named ``crys_*`` mirror the C ABI in ``include/crystal.h`` one for one and
only marshal arguments (tensors -> device pointers, the current torch stream -> a
cudaStream_t); every step of every operator runs in the library's CUDA kernels.
PyTorch supplies device memory and streams.  There is no CPU fallback: importing the
operators without the built library raises.

Convenience wrappers (``select``, ``project``, ``HashTable``, ``probe_aggregate``,
``sort``, ``make_table``, ``make_plan``, ``run_plan``) allocate outputs and scratch with
torch and call the ``crys_*`` functions; ``starschema`` (resident star schema, tagged
shared scans, graph-replayed launches) and ``server`` (continuous batching) build on them.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcrystal.so")

OK, EINVAL, ENOMEM, EFULL, ETIMEOUT, ECUDA = 0, -1, -2, -3, -4, -5
DEV_TIMEOUT, DEV_TABLE_FULL, DEV_BAD_KEY, DEV_DUP_KEY, DEV_BAD_GROUP, DEV_BOUNDS = 1, 2, 4, 8, 16, 32
PROJ_LINEAR, PROJ_SIGMOID = 0, 1
AGG_A, AGG_A_MUL_B, AGG_A_SUB_B, AGG_A_ADD_B = 0, 1, 2, 3
AGG_OPS = {"sum": AGG_A, "mul": AGG_A_MUL_B, "sub": AGG_A_SUB_B, "add": AGG_A_ADD_B}
MAX_COLS, MAX_PREDS, MAX_JOINS, MAX_PLANS, MAX_FIELD_PREDS = 16, 8, 4, 32, 2
ACCUMULATE = 1
TAG_ANNOTATE = 2
HASH_MULT, HASH_IDENT, HASH_DIRECT = 0, 1, 2
OP_SELECT, OP_PROJECT, OP_PROBE, OP_PLAN, OP_SHARED_SCAN, OP_SORT, OP_TAGGED_SCAN = range(7)
NUM_OPS = 7
OP_NAMES = ["select", "project", "probe", "plan", "shared_scan", "sort", "tagged_scan"]


class CrystalError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {status} ({strerror(status)})")
        self.status = status


# ---------------------------------------------------------------- C structures

class crys_hash(C.Structure):
    _fields_ = [("slots", C.c_void_p), ("capacity", C.c_int64), ("kind", C.c_int32)]


class crys_pred(C.Structure):
    _fields_ = [("col", C.c_void_p), ("lo", C.c_int32), ("hi", C.c_int32)]


class crys_table(C.Structure):
    _fields_ = [("cols", C.c_void_p * MAX_COLS), ("n_cols", C.c_int32), ("n_rows", C.c_int64)]


class crys_col_pred(C.Structure):
    _fields_ = [("col", C.c_int32), ("lo", C.c_int32), ("hi", C.c_int32)]


class crys_field_pred(C.Structure):
    _fields_ = [("shift", C.c_int32), ("bits", C.c_int32), ("lo", C.c_int32), ("hi", C.c_int32)]


class crys_join(C.Structure):
    _fields_ = [("fk_col", C.c_int32), ("ht", crys_hash), ("group_card", C.c_int32),
                ("group_shift", C.c_int32), ("group_bits", C.c_int32), ("n_preds", C.c_int32),
                ("preds", crys_field_pred * MAX_FIELD_PREDS)]


class crys_plan(C.Structure):
    _fields_ = [("n_preds", C.c_int32), ("preds", crys_col_pred * MAX_PREDS),
                ("n_joins", C.c_int32), ("joins", crys_join * MAX_JOINS),
                ("agg_op", C.c_int32), ("agg_a", C.c_int32), ("agg_b", C.c_int32),
                ("d_sums", C.c_void_p), ("d_counts", C.c_void_p)]


_lib = None


def lib():
    """The loaded operator library.  Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "(there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        p, i64, i32, sz = C.c_void_p, C.c_int64, C.c_int32, C.POINTER(C.c_size_t)
        L.crys_strerror.argtypes = [C.c_int]
        L.crys_strerror.restype = C.c_char_p
        L.crys_device_errors.argtypes = [C.POINTER(C.c_int32), C.c_int, p]
        L.crys_launch_count.restype = i64
        L.crys_debug_stall.argtypes = [C.c_int, i32, i64]
        L.crys_select.argtypes = [p, i64, i32, i32, p, p, C.c_int, p, sz, p]
        L.crys_select_static.argtypes = [p, i64, i32, i32, p, p, p]
        L.crys_select_strawman.argtypes = [p, i64, i32, i32, p, p, p, sz, p]
        L.crys_project.argtypes = [p, p, i64, C.c_float, C.c_float, C.c_int, p, p]
        L.crys_hash_init.argtypes = [C.POINTER(crys_hash), p]
        L.crys_hash_build.argtypes = [p, p, i64, C.POINTER(crys_pred), i32, C.POINTER(crys_hash), p]
        L.crys_probe_aggregate.argtypes = [p, p, i64, C.POINTER(crys_hash), p, p, p]
        L.crys_sort.argtypes = [p, p, p, p, i64, p, sz, p]
        L.crys_sort_msb.argtypes = [p, p, p, p, i64, p, sz, p]
        L.crys_join_partitioned.argtypes = [p, p, i64, p, p, i64, p, p, p, sz, p]
        L.crys_plan_groups.argtypes = [C.POINTER(crys_plan), C.POINTER(C.c_int64)]
        L.crys_pack_fields.argtypes = [C.POINTER(C.c_void_p), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                       i32, i64, p, p]
        L.crys_run_plan.argtypes = [C.POINTER(crys_table), C.POINTER(crys_plan), p]
        L.crys_run_plans.argtypes = [C.POINTER(crys_table), C.POINTER(crys_plan), i32, i64, i64,
                                     C.c_int, p]
        L.crys_run_plans_tagged_bytes.argtypes = [C.POINTER(crys_table), C.POINTER(crys_plan), i32,
                                                  C.POINTER(C.c_int64)]
        L.crys_run_plans_tagged.argtypes = [C.POINTER(crys_table), C.POINTER(crys_plan), i32, i64, i64,
                                            C.c_int, p, i64, p]
        L.crys_tagged_block_bytes.argtypes = [C.POINTER(C.c_int64)]
        L.crys_tagged_prepare.argtypes = [C.POINTER(crys_table), C.POINTER(crys_plan), i32, i64, i64, C.c_int,
                                          C.POINTER(C.c_int32), i32, p, i64, p]
        L.crys_tagged_launch.argtypes = [p, p]
        L.crys_tile_variants.argtypes = [C.c_int, C.POINTER(C.c_int32), C.POINTER(C.c_int32), i32]
        L.crys_set_tile.argtypes = [C.c_int, i32]
        L.crys_get_tile.argtypes = [C.c_int]
        for fn in ("crys_device_errors", "crys_debug_stall", "crys_select", "crys_select_static", "crys_select_strawman",
                   "crys_project", "crys_hash_init",
                   "crys_hash_build", "crys_probe_aggregate", "crys_sort", "crys_sort_msb",
                   "crys_join_partitioned", "crys_plan_groups",
                   "crys_pack_fields",
                   "crys_run_plan", "crys_run_plans", "crys_run_plans_tagged_bytes",
                   "crys_run_plans_tagged", "crys_tagged_block_bytes", "crys_tagged_prepare",
                   "crys_tagged_launch", "crys_tile_variants", "crys_set_tile",
                   "crys_get_tile"):
            getattr(L, fn).restype = C.c_int
        _lib = L
    return _lib


def strerror(status: int) -> str:
    return lib().crys_strerror(status).decode()


def _check(status: int, where: str) -> None:
    if status != OK:
        raise CrystalError(status, where)


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_cuda:
        raise ValueError("device tensor expected")
    return t.data_ptr()


def _stream(stream=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


# ---------------------------------------------------------------- crys_* (same names)

def crys_device_errors(clear: bool = True, stream=None) -> int:
    flags = C.c_int32(0)
    _check(lib().crys_device_errors(C.byref(flags), int(clear), _stream(stream)), "crys_device_errors")
    return flags.value


def crys_launch_count() -> int:
    return int(lib().crys_launch_count())


def crys_debug_stall(op: int, first_tile: int, wait_limit_ns: int) -> None:
    """Test hook: the next order-preserving select or sort starts its tile ids at
    first_tile (earlier tiles never publish) and bounds its look-back waits."""
    _check(lib().crys_debug_stall(op, first_tile, wait_limit_ns), "crys_debug_stall")


def crys_select(x, n: int, lo: int, hi: int, out, d_count, order_preserving: int = 0,
                d_temp=None, temp_bytes: int | None = None, stream=None) -> int:
    """Returns the scratch size when d_temp is None and temp_bytes is requested (-1)."""
    if d_temp is None and temp_bytes == -1:
        size = C.c_size_t(0)
        _check(lib().crys_select(None, n, lo, hi, None, None, order_preserving, None, C.byref(size), None),
               "crys_select")
        return size.value
    tb = C.c_size_t(temp_bytes if temp_bytes is not None else 0)
    _check(lib().crys_select(_ptr(x), n, lo, hi, _ptr(out), _ptr(d_count), order_preserving,
                             _ptr(d_temp), C.byref(tb) if d_temp is not None else None, _stream(stream)),
           "crys_select")
    return 0


def crys_select_static(x, n: int, lo: int, hi: int, out, d_count, stream=None) -> None:
    """Order-preserving selection whose scratch is the library's static device array
    (no allocation on the call path; n <= 2^25)."""
    _check(lib().crys_select_static(_ptr(x), n, lo, hi, _ptr(out), _ptr(d_count), _stream(stream)),
           "crys_select_static")


def crys_select_strawman(x, n: int, lo: int, hi: int, out, d_count, d_temp=None, temp_bytes: int | None = None,
                         stream=None) -> int:
    """The independent-threads selection (ablation).  Returns the scratch size when
    d_temp is None and temp_bytes is -1."""
    if d_temp is None and temp_bytes == -1:
        size = C.c_size_t(0)
        _check(lib().crys_select_strawman(None, n, lo, hi, None, None, None, C.byref(size), None),
               "crys_select_strawman")
        return size.value
    tb = C.c_size_t(temp_bytes if temp_bytes is not None else 0)
    _check(lib().crys_select_strawman(_ptr(x), n, lo, hi, _ptr(out), _ptr(d_count), _ptr(d_temp), C.byref(tb),
                                      _stream(stream)), "crys_select_strawman")
    return 0


def crys_project(x1, x2, n: int, a: float, b: float, op: int, y, stream=None) -> None:
    _check(lib().crys_project(_ptr(x1), _ptr(x2), n, a, b, op, _ptr(y), _stream(stream)), "crys_project")


def crys_hash_init(ht: crys_hash, stream=None) -> None:
    _check(lib().crys_hash_init(C.byref(ht), _stream(stream)), "crys_hash_init")


def crys_hash_build(keys, vals, n: int, filters: list, ht: crys_hash, stream=None) -> None:
    arr = (crys_pred * max(1, len(filters)))(*[crys_pred(_ptr(c), lo, hi) for c, lo, hi in filters])
    _check(lib().crys_hash_build(_ptr(keys), _ptr(vals), n, arr if filters else None, len(filters),
                                 C.byref(ht), _stream(stream)), "crys_hash_build")


def crys_probe_aggregate(fk, payload, n: int, ht: crys_hash, d_sum, d_matches=None, stream=None) -> None:
    _check(lib().crys_probe_aggregate(_ptr(fk), _ptr(payload), n, C.byref(ht), _ptr(d_sum),
                                      _ptr(d_matches), _stream(stream)), "crys_probe_aggregate")


def crys_sort(keys_in, vals_in, keys_out, vals_out, n: int, d_temp=None, temp_bytes: int | None = None,
              stream=None) -> int:
    if d_temp is None and temp_bytes == -1:
        size = C.c_size_t(0)
        _check(lib().crys_sort(None, None, None, None, n, None, C.byref(size), None), "crys_sort")
        return size.value
    tb = C.c_size_t(temp_bytes if temp_bytes is not None else 0)
    _check(lib().crys_sort(_ptr(keys_in), _ptr(vals_in), _ptr(keys_out), _ptr(vals_out), n,
                           _ptr(d_temp), C.byref(tb), _stream(stream)), "crys_sort")
    return 0


def crys_sort_msb(keys_in, vals_in, keys_out, vals_out, n: int, d_temp=None, temp_bytes: int | None = None,
                  stream=None) -> int:
    """MSB radix sort (unstable).  Returns the scratch size when d_temp is None and
    temp_bytes is -1."""
    if d_temp is None and temp_bytes == -1:
        size = C.c_size_t(0)
        _check(lib().crys_sort_msb(None, None, None, None, n, None, C.byref(size), None), "crys_sort_msb")
        return size.value
    tb = C.c_size_t(temp_bytes if temp_bytes is not None else 0)
    _check(lib().crys_sort_msb(_ptr(keys_in), _ptr(vals_in), _ptr(keys_out), _ptr(vals_out), n,
                               _ptr(d_temp), C.byref(tb), _stream(stream)), "crys_sort_msb")
    return 0


def crys_join_partitioned(bkeys, bvals, nb: int, fk, payload, np_: int, d_sum, d_matches=None, d_temp=None,
                          temp_bytes: int | None = None, stream=None) -> int:
    """Radix-partitioned join + SUM(payload * value).  Returns the scratch size when d_temp
    is None and temp_bytes is -1."""
    if d_temp is None and temp_bytes == -1:
        size = C.c_size_t(0)
        _check(lib().crys_join_partitioned(None, None, nb, None, None, np_, None, None, None, C.byref(size), None),
               "crys_join_partitioned")
        return size.value
    tb = C.c_size_t(temp_bytes if temp_bytes is not None else 0)
    _check(lib().crys_join_partitioned(_ptr(bkeys), _ptr(bvals), nb, _ptr(fk), _ptr(payload), np_, _ptr(d_sum),
                                       _ptr(d_matches), _ptr(d_temp), C.byref(tb), _stream(stream)),
           "crys_join_partitioned")
    return 0


def crys_plan_groups(plan: crys_plan) -> int:
    g = C.c_int64(0)
    _check(lib().crys_plan_groups(C.byref(plan), C.byref(g)), "crys_plan_groups")
    return g.value


def crys_pack_fields(cols: list, shifts: list, bits: list, n: int, out, stream=None) -> None:
    k = len(cols)
    carr = (C.c_void_p * max(1, k))(*[_ptr(c) for c in cols])
    sarr = (C.c_int32 * max(1, k))(*shifts)
    barr = (C.c_int32 * max(1, k))(*bits)
    _check(lib().crys_pack_fields(carr, sarr, barr, k, n, _ptr(out), _stream(stream)), "crys_pack_fields")


def crys_run_plan(fact: crys_table, plan: crys_plan, stream=None) -> None:
    _check(lib().crys_run_plan(C.byref(fact), C.byref(plan), _stream(stream)), "crys_run_plan")


def crys_run_plans(fact: crys_table, plans, row_begin: int, row_end: int, flags: int = 0,
                   stream=None) -> None:
    arr = (crys_plan * max(1, len(plans)))(*plans)
    _check(lib().crys_run_plans(C.byref(fact), arr, len(plans), row_begin, row_end, flags,
                                _stream(stream)), "crys_run_plans")


def crys_run_plans_tagged_bytes(fact: crys_table, plans) -> int:
    """Scratch bytes of the query bitmaps of a batch; 0 when it cannot be tagged."""
    arr = (crys_plan * max(1, len(plans)))(*plans)
    out = C.c_int64(0)
    _check(lib().crys_run_plans_tagged_bytes(C.byref(fact), arr, len(plans), C.byref(out)),
           "crys_run_plans_tagged_bytes")
    return out.value


def crys_run_plans_tagged(fact: crys_table, plans, row_begin: int, row_end: int, flags: int = 0,
                          scratch=None, scratch_bytes: int = 0, stream=None) -> None:
    arr = (crys_plan * max(1, len(plans)))(*plans)
    _check(lib().crys_run_plans_tagged(C.byref(fact), arr, len(plans), row_begin, row_end, flags,
                                       _ptr(scratch), scratch_bytes, _stream(stream)),
           "crys_run_plans_tagged")


def crys_tagged_block_bytes() -> int:
    out = C.c_int64(0)
    _check(lib().crys_tagged_block_bytes(C.byref(out)), "crys_tagged_block_bytes")
    return out.value


def crys_tagged_prepare(fact: crys_table, plans, row_begin: int, row_end: int, flags: int, zero_plans,
                        scratch, scratch_bytes: int, host_block: int) -> int:
    """Fills the host argument block at address `host_block`; returns the status (no raise:
    CRYS_EINVAL means the batch cannot use the replayable launch)."""
    arr = (crys_plan * max(1, len(plans)))(*plans)
    z = (C.c_int32 * max(1, len(zero_plans)))(*zero_plans)
    return lib().crys_tagged_prepare(C.byref(fact), arr, len(plans), row_begin, row_end, flags, z,
                                     len(zero_plans), _ptr(scratch), scratch_bytes, host_block)


def crys_tagged_launch(dev_block, stream=None) -> None:
    _check(lib().crys_tagged_launch(_ptr(dev_block), _stream(stream)), "crys_tagged_launch")


def crys_tile_variants(op: int) -> list:
    t = (C.c_int32 * 16)()
    i = (C.c_int32 * 16)()
    n = lib().crys_tile_variants(op, t, i, 16)
    if n < 0:
        raise CrystalError(n, "crys_tile_variants")
    return [(t[k], i[k]) for k in range(n)]


def crys_set_tile(op: int, variant: int) -> None:
    _check(lib().crys_set_tile(op, variant), "crys_set_tile")


def crys_get_tile(op: int) -> int:
    return int(lib().crys_get_tile(op))


# ---------------------------------------------------------------- conveniences

def _dev(t: torch.Tensor) -> torch.device:
    return t.device


def check_device_errors(stream=None) -> None:
    flags = crys_device_errors(clear=True, stream=stream)
    if flags:
        names = [n for n, b in [("timeout", DEV_TIMEOUT), ("table_full", DEV_TABLE_FULL),
                                ("bad_key", DEV_BAD_KEY), ("dup_key", DEV_DUP_KEY),
                                ("bad_group", DEV_BAD_GROUP), ("bounds", DEV_BOUNDS)] if flags & b]
        raise RuntimeError(f"device error flags 0x{flags:x}: {', '.join(names)}")


def scratch(nbytes: int, device) -> torch.Tensor:
    """Device scratch buffer of at least nbytes (256-byte aligned by the caching allocator)."""
    return torch.empty(max(1, nbytes), dtype=torch.uint8, device=device)


def select(x: torch.Tensor, lo: int, hi: int, order_preserving: bool = False, stream=None):
    """Values of x with lo <= x <= hi (compacted).  Synchronises to read the count."""
    n = x.numel()
    out = torch.empty(max(1, n), dtype=torch.int32, device=x.device)
    count = torch.zeros(1, dtype=torch.int64, device=x.device)
    temp, tb = None, None
    if order_preserving:
        tb = crys_select(None, n, lo, hi, None, None, 1, None, -1)
        temp = scratch(tb, x.device)
    crys_select(x, n, lo, hi, out, count, int(order_preserving), temp, tb, stream)
    c = int(count.item())
    return out[:c]


def project(x1: torch.Tensor, x2: torch.Tensor, a: float = 2.0, b: float = 3.0, op: int = PROJ_LINEAR,
            out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    y = torch.empty_like(x1) if out is None else out
    crys_project(x1, x2, x1.numel(), a, b, op, y, stream)
    return y


def capacity_for(rows: int, kind: int = 0) -> int:
    """Capacity for `rows` keys: a power of two at most 50% full for multiplicative
    hashing; a power of two of at least `rows` slots for identity hashing of dense keys;
    exactly `rows` slots for a direct table of the keys 0..rows-1."""
    if kind == HASH_DIRECT:
        return max(1, rows)
    need = 2 * rows if kind == HASH_MULT else rows
    cap = 2
    while cap < need:
        cap *= 2
    return cap


class HashTable:
    """A device hash table (caller-owned slot array) and its crys_hash view."""

    def __init__(self, capacity: int, device, kind: int = HASH_MULT):
        if kind == HASH_DIRECT:
            if capacity < 1:
                raise ValueError("a direct table needs capacity >= 1")
        elif capacity < 2 or capacity & (capacity - 1):
            raise ValueError("capacity must be a power of two >= 2")
        self.slots = torch.empty(capacity, dtype=torch.int64, device=device)
        self.capacity = capacity
        self.kind = kind
        self.struct = crys_hash(self.slots.data_ptr(), capacity, kind)

    @classmethod
    def build(cls, keys: torch.Tensor, vals: torch.Tensor | None = None, filters=(), capacity=None,
              stream=None, kind: int = HASH_MULT) -> "HashTable":
        ht = cls(capacity or capacity_for(keys.numel(), kind), keys.device, kind)
        crys_hash_init(ht.struct, stream)
        crys_hash_build(keys, vals, keys.numel(), list(filters), ht.struct, stream)
        return ht

    @property
    def nbytes(self) -> int:
        return self.capacity * 8


def probe_aggregate(fk: torch.Tensor, payload: torch.Tensor, ht: HashTable, stream=None):
    """(SUM(payload * value), matches) as int64 device tensors of one element."""
    out = torch.zeros(2, dtype=torch.int64, device=fk.device)
    crys_probe_aggregate(fk, payload, fk.numel(), ht.struct, out[0:1], out[1:2], stream)
    return out[0:1], out[1:2]


def sort(keys: torch.Tensor, vals: torch.Tensor, stream=None):
    n = keys.numel()
    ko = torch.empty_like(keys)
    vo = torch.empty_like(vals)
    tb = crys_sort(None, None, None, None, n, None, -1)
    temp = scratch(tb, keys.device)
    crys_sort(keys, vals, ko, vo, n, temp, tb, stream)
    return ko, vo


def sort_msb(keys: torch.Tensor, vals: torch.Tensor, stream=None):
    """Unstable MSB radix sort: keys ascending (signed), equal keys' values in any order."""
    n = keys.numel()
    ko = torch.empty_like(keys)
    vo = torch.empty_like(vals)
    tb = crys_sort_msb(None, None, None, None, n, None, -1)
    temp = scratch(tb, keys.device)
    crys_sort_msb(keys, vals, ko, vo, n, temp, tb, stream)
    return ko, vo


def join_partitioned(bkeys: torch.Tensor, bvals: torch.Tensor, fk: torch.Tensor, payload: torch.Tensor,
                     stream=None):
    """(SUM(payload * value), matches) of the radix-partitioned join, int64 device tensors."""
    out = torch.zeros(2, dtype=torch.int64, device=fk.device)
    tb = crys_join_partitioned(None, None, bkeys.numel(), None, None, fk.numel(), None, None, None, -1)
    temp = scratch(tb, fk.device)
    crys_join_partitioned(bkeys, bvals, bkeys.numel(), fk, payload, fk.numel(), out[0:1], out[1:2], temp, tb,
                          stream)
    return out[0:1], out[1:2]


def make_table(cols: list) -> crys_table:
    t = crys_table()
    if len(cols) > MAX_COLS:
        raise ValueError("too many columns")
    n = cols[0].numel() if cols else 0
    for i, c in enumerate(cols):
        if c.dtype != torch.int32 or c.numel() != n or not c.is_contiguous():
            raise ValueError("fact columns must be contiguous int32 of equal length")
        t.cols[i] = c.data_ptr()
    t.n_cols = len(cols)
    t.n_rows = n
    return t


def make_plan(preds, joins, agg, sums: torch.Tensor, counts: torch.Tensor | None) -> crys_plan:
    """preds: [(col, lo, hi)]; joins: [(fk_col, HashTable, group_card)] for tables whose
    value is the group code, or [(fk_col, HashTable, group_card, (group_shift, group_bits),
    [(shift, bits, lo, hi), ...])] for tables whose value packs attribute fields;
    agg: (op, a, b)."""
    p = crys_plan()
    if len(preds) > MAX_PREDS or len(joins) > MAX_JOINS:
        raise ValueError("too many predicates or joins")
    p.n_preds = len(preds)
    for i, (c, lo, hi) in enumerate(preds):
        p.preds[i] = crys_col_pred(c, lo, hi)
    p.n_joins = len(joins)
    for i, jn in enumerate(joins):
        fk, ht, card = jn[0], jn[1], jn[2]
        js = crys_join()
        js.fk_col, js.ht, js.group_card = fk, ht.struct, card
        if len(jn) > 3:
            js.group_shift, js.group_bits = jn[3]
            fps = list(jn[4])
            if len(fps) > MAX_FIELD_PREDS:
                raise ValueError("too many dimension predicates")
            js.n_preds = len(fps)
            for k, (sh, bi, lo, hi) in enumerate(fps):
                js.preds[k] = crys_field_pred(sh, bi, lo, hi)
        p.joins[i] = js
    op, a, b = agg
    p.agg_op = AGG_OPS[op] if isinstance(op, str) else op
    p.agg_a = a
    p.agg_b = b if b is not None else 0
    p.d_sums = sums.data_ptr()
    p.d_counts = counts.data_ptr() if counts is not None else None
    return p


def plan_groups(joins) -> int:
    g = 1
    for jn in joins:
        card = jn[2]
        if card > 0:
            g *= card
    return g


def run_plan(fact_cols: list, preds, joins, agg, stream=None):
    """One select-join-aggregate query -> (sums, counts) device int64 tensors."""
    dev = fact_cols[0].device
    g = plan_groups(joins)
    sums = torch.empty(g, dtype=torch.int64, device=dev)
    counts = torch.empty(g, dtype=torch.int64, device=dev)
    crys_run_plan(make_table(fact_cols), make_plan(preds, joins, agg, sums, counts), stream)
    return sums, counts
