"""The allocation-free selection entry point (crys_select_static) against the regular
order-preserving selection (crys_select with caller scratch), through the C ABI.

crys_select_static serves callers that cannot allocate device memory while a query runs
(executors inside a host process that owns a fixed device pool, pipelines that forbid
allocation after start-up); its scratch is a static device array shared by all calls.
This file is collected last so that a failure here comes after every other test ran."""
import ctypes as C

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
    return crys


def _regular(crys, x, lo, hi):
    n = x.numel()
    out = torch.empty(max(1, n), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    tb = crys.crys_select(None, n, lo, hi, None, None, 1, None, -1)
    temp = crys.scratch(tb, "cuda")
    crys.crys_select(x, n, lo, hi, out, cnt, 1, temp, tb)
    c = int(cnt.item())
    return out[:c].cpu().numpy()


def _static(crys, x, lo, hi):
    n = x.numel()
    out = torch.full((max(1, n),), -7, dtype=torch.int32, device="cuda")
    cnt = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    rc = crys.lib().crys_select_static(C.c_void_p(x.data_ptr()), n, lo, hi, C.c_void_p(out.data_ptr()),
                                       C.c_void_p(cnt.data_ptr()),
                                       C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == crys.OK, crys.strerror(rc)
    c = int(cnt.item())
    return out[:c].cpu().numpy()


def test_static_select_matches_regular_twice_in_a_row(crys):
    # two calls in a row on the shared static scratch: a large one, then a smaller one
    # (stale look-back words of the first must not leak into the second)
    cases = [(3_000_017, datagen.select_threshold(0.5)), (777_777, datagen.select_threshold(0.2))]
    for i, (n, hi) in enumerate(cases):
        x = torch.from_numpy(datagen.uniform_i32(50 + i, datagen.STREAMS["sel.x"], n, 0, I32_MAX)).cuda()
        ref = _regular(crys, x, I32_MIN, hi)
        got = _static(crys, x, I32_MIN, hi)
        assert got.size == ref.size and np.array_equal(got, ref), i


def test_static_select_limits(crys):
    L = crys.lib()
    big = (1 << 25) + 1
    assert L.crys_select_static(None, big, 0, 1, None, None, None) == crys.EINVAL
    x = torch.arange(1 << 25, dtype=torch.int32, device="cuda")      # exactly the maximum
    got = _static(crys, x, 100, 1 << 24)
    assert np.array_equal(got, np.arange(100, (1 << 24) + 1, dtype=np.int32))


def test_static_select_empty_inputs_then_a_normal_call(crys):
    # n = 0 and an empty range (lo > hi) return no rows; the empty range clears the static
    # array's used part, and the next call on the array is still exact
    empty = torch.empty(0, dtype=torch.int32, device="cuda")
    assert _static(crys, empty, 0, 10).size == 0
    x = torch.from_numpy(datagen.uniform_i32(61, datagen.STREAMS["sel.x"], 100_003, 0, I32_MAX)).cuda()
    assert _static(crys, x, 10, 5).size == 0
    hi = datagen.select_threshold(0.4)
    assert np.array_equal(_static(crys, x, I32_MIN, hi), _regular(crys, x, I32_MIN, hi))


def test_static_select_left_no_device_error(crys):
    assert crys.crys_device_errors(clear=True) == 0
