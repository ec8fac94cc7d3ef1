"""Device twin of the seeded input generator (datagen/gen.cu -> datagen/libcrysgen.so):
fills torch CUDA tensors with exactly the values datagen/__init__.py defines.  Input
generation only."""
from __future__ import annotations

import ctypes as C
import os

import torch

from . import STREAMS, SS_DIMS, SS_FACT_COLS, SS_FACT_RANGES, Q1_DIM_ROWS, ss_dim_scale

_LIB = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libcrysgen.so")
_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB):
            raise RuntimeError(f"{_LIB} is missing: build it with __graft_entry__.build()")
        L = C.CDLL(_LIB)
        u64, i64, i32, p = C.c_uint64, C.c_int64, C.c_int32, C.c_void_p
        L.dg_uniform_i32.argtypes = [u64, u64, i64, i64, i32, i32, p, p]
        L.dg_uniform_f32.argtypes = [u64, u64, i64, i64, p, p]
        L.dg_bits_i32.argtypes = [u64, u64, i64, i64, p, p]
        L.dg_perm_i32.argtypes = [u64, u64, i64, i64, i64, p, p]
        for f in ("dg_uniform_i32", "dg_uniform_f32", "dg_bits_i32", "dg_perm_i32"):
            getattr(L, f).restype = C.c_int
        _lib = L
    return _lib


def _s():
    return torch.cuda.current_stream().cuda_stream


def _ok(rc, what):
    if rc != 0:
        raise RuntimeError(f"{what} failed ({rc})")


def uniform_i32(seed, stream, n, lo, hi, device="cuda", start=0, out=None):
    out = torch.empty(n, dtype=torch.int32, device=device) if out is None else out
    _ok(lib().dg_uniform_i32(seed, stream, start, n, lo, hi, out.data_ptr(), _s()), "dg_uniform_i32")
    return out


def uniform_f32(seed, stream, n, device="cuda", start=0, out=None):
    out = torch.empty(n, dtype=torch.float32, device=device) if out is None else out
    _ok(lib().dg_uniform_f32(seed, stream, start, n, out.data_ptr(), _s()), "dg_uniform_f32")
    return out


def bits_i32(seed, stream, n, device="cuda", start=0, out=None):
    out = torch.empty(n, dtype=torch.int32, device=device) if out is None else out
    _ok(lib().dg_bits_i32(seed, stream, start, n, out.data_ptr(), _s()), "dg_bits_i32")
    return out


def perm_i32(seed, stream, n, device="cuda", start=0, count=None, out=None):
    count = n - start if count is None else count
    out = torch.empty(count, dtype=torch.int32, device=device) if out is None else out
    _ok(lib().dg_perm_i32(seed, stream, n, start, count, out.data_ptr(), _s()), "dg_perm_i32")
    return out


def q1_tables(seed, n_fact, device="cuda"):
    fact = {
        "fk": uniform_i32(seed, STREAMS["q1.fk"], n_fact, 0, Q1_DIM_ROWS - 1, device),
        "a": uniform_i32(seed, STREAMS["q1.a"], n_fact, 1, 50, device),
        "b": uniform_i32(seed, STREAMS["q1.b"], n_fact, 0, 10, device),
        "c": uniform_i32(seed, STREAMS["q1.c"], n_fact, 1, 100000, device),
    }
    dim = {
        "key": perm_i32(seed, STREAMS["q1.dim_key"], Q1_DIM_ROWS, device),
        "yr": (torch.arange(Q1_DIM_ROWS, device=device) % 7).to(torch.int32),
    }
    return {"fact": fact, "dim": dim}


def ss_fact_col(seed, name, n, device="cuda", dim_scale=1.0):
    lo, hi = SS_FACT_RANGES[name]
    if name.startswith("fk_"):
        dim = {"fk_date": "date", "fk_supp": "supp", "fk_cust": "cust", "fk_part": "part"}[name]
        hi = ss_dim_scale(SS_DIMS[dim]["rows"], dim_scale) - 1
    return uniform_i32(seed, STREAMS["ss." + name], n, lo, hi, device)


def ss_dimension(seed, dim, device="cuda", dim_scale=1.0):
    spec = SS_DIMS[dim]
    rows = ss_dim_scale(spec["rows"], dim_scale)
    out = {"key": perm_i32(seed, STREAMS[f"ss.{dim}.key"], rows, device)}
    for attr, card in spec["attrs"].items():
        out[attr] = uniform_i32(seed, STREAMS[f"ss.{dim}.{attr}"], rows, 0, card - 1, device)
    return out


def ss_tables(seed, n_fact, device="cuda", dim_scale=1.0):
    fact = {c: ss_fact_col(seed, c, n_fact, device, dim_scale) for c in SS_FACT_COLS}
    dims = {d: ss_dimension(seed, d, device, dim_scale) for d in SS_DIMS}
    return {"fact": fact, "dims": dims}
