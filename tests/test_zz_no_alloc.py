"""The allocation-free sort entry point, through the C ABI.

tigas_sort_pairs_u64_noalloc exists for callers that cannot let the library
call cudaMalloc (they manage all device memory themselves, or cannot take the
synchronisation an allocation may cause); it keeps its scratch in one fixed
device array.  This file checks:
  - that a call allocates no device memory (free memory unchanged);
  - that it matches tigas_sort_pairs_u64 on two calls in a row, so the second
    call runs on scratch the first one left behind;
  - that tigas_sort_noalloc_check reports OK after normal sorts, reports the
    run-out look-back wait the test hook forces (the call itself is
    asynchronous and cannot), clears it, and that the next sort is still
    correct;
  - the size limit.
The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2605_08699_b300 as tg  # noqa: E402
from paper_2605_08699_b300 import tigas as tb  # noqa: E402

MAX_PAIRS = 1 << 20


def _inputs(n, seed, distinct=None):
    rng = np.random.default_rng(seed)
    if distinct:
        keys = rng.integers(0, distinct, size=n, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15)
    else:
        keys = rng.integers(0, 2 ** 63, size=n, dtype=np.uint64)
    vals = rng.permutation(n).astype(np.uint32)
    dev = torch.device("cuda:0")
    return keys, vals, torch.from_numpy(keys.view(np.int64)).to(dev), torch.from_numpy(vals.view(np.int32)).to(dev)


def _sort(fn_name, kin, vin, n, b0, b1, kout=None, vout=None):
    lib = tg.load_library()
    if kout is None:
        kout, vout = torch.empty_like(kin), torch.empty_like(vin)
    st = getattr(lib, fn_name)(kin.data_ptr(), vin.data_ptr(), kout.data_ptr(), vout.data_ptr(), ctypes.c_uint64(n),
                               b0, b1, None)
    assert st == tb.OK, tg.last_error()
    torch.cuda.synchronize()
    return kout.cpu().numpy(), vout.cpu().numpy()


def _check():
    return tg.load_library().tigas_sort_noalloc_check(None)


def test_noalloc_sort_allocates_no_device_memory():
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    # warm-up: the first call on the device loads the module and looks up the scratch address
    _, _, kw, vw = _inputs(4096, 7)
    _sort("tigas_sort_pairs_u64_noalloc", kw, vw, 4096, 0, 45)
    _, _, kin, vin = _inputs(MAX_PAIRS, 8)
    kout, vout = torch.empty_like(kin), torch.empty_like(vin)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        _sort("tigas_sort_pairs_u64_noalloc", kin, vin, MAX_PAIRS, 0, 64, kout, vout)
    assert _check() == tb.OK, tg.last_error()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_sort_matches_allocating_sort_twice_in_a_row():
    assert torch.cuda.is_available()
    cases = [(MAX_PAIRS, 0, 45, 1000), (300_001, 3, 40, None)]   # two calls, different sizes and bits
    for seed, (n, b0, b1, distinct) in enumerate(cases):
        keys, vals, kin, vin = _inputs(n, 100 + seed, distinct)
        k_ref, v_ref = _sort("tigas_sort_pairs_u64", kin, vin, n, b0, b1)
        k_new, v_new = _sort("tigas_sort_pairs_u64_noalloc", kin, vin, n, b0, b1)
        # integer outputs: bit-exact (the tolerance of every integer parity test)
        assert np.array_equal(k_new, k_ref) and np.array_equal(v_new, v_ref)
        # and both are the stable order of the selected key bits
        sub = (keys >> np.uint64(b0)) & np.uint64((1 << (b1 - b0)) - 1)
        assert np.array_equal(v_new.view(np.uint32), vals[np.argsort(sub, kind="stable")])
    # no look-back wait of these sorts ran out
    assert _check() == tb.OK, tg.last_error()


def test_noalloc_check_reports_a_run_out_wait_once_and_the_sort_stays_correct():
    lib = tg.load_library()
    assert _check() == tb.OK, tg.last_error()
    # the hook's one scatter CTA waits on a chunk nobody publishes: each wait gives up
    # after the spin limit and the run-out is recorded in the sticky word
    assert lib.tigas_debug_sort_noalloc_wait_timeout(2048, None) == tb.OK, tg.last_error()
    assert _check() == tb.ERR_TIMEOUT
    assert "ran out" in tg.last_error()
    assert _check() == tb.OK, tg.last_error()   # read and cleared
    # the device and the shared scratch stay usable
    keys, vals, kin, vin = _inputs(65_537, 11)
    k_ref, v_ref = _sort("tigas_sort_pairs_u64", kin, vin, 65_537, 0, 64)
    k_new, v_new = _sort("tigas_sort_pairs_u64_noalloc", kin, vin, 65_537, 0, 64)
    assert np.array_equal(k_new, k_ref) and np.array_equal(v_new, v_ref)
    assert _check() == tb.OK, tg.last_error()
    assert lib.tigas_debug_sort_noalloc_wait_timeout(0, None) == tb.ERR_INVALID


def test_noalloc_sort_rejects_sizes_beyond_its_maximum():
    lib = tg.load_library()
    st = lib.tigas_sort_pairs_u64_noalloc(None, None, None, None, ctypes.c_uint64(MAX_PAIRS + 1), 0, 64, None)
    assert st == tb.ERR_INVALID
    assert "1048576" in tg.last_error()
