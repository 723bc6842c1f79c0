"""The allocation-free sort entry point, through the C ABI.

tigas_sort_pairs_u64_noalloc exists for callers that cannot let the library
call cudaMalloc (they manage all device memory themselves, or cannot take the
synchronisation an allocation may cause); it keeps its scratch in one fixed
device array.  This test checks it against tigas_sort_pairs_u64 on two calls
in a row, so the second call runs on scratch the first one left behind.  The
file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2605_08699_b300 as tg  # noqa: E402
from paper_2605_08699_b300 import tigas as tb  # noqa: E402

MAX_PAIRS = 1 << 20


def _sort(fn_name, kin, vin, n, b0, b1):
    lib = tg.load_library()
    kout, vout = torch.empty_like(kin), torch.empty_like(vin)
    fn = getattr(lib, fn_name)
    st = fn(kin.data_ptr(), vin.data_ptr(), kout.data_ptr(), vout.data_ptr(), ctypes.c_uint64(n), b0, b1, None)
    assert st == tb.OK, tg.last_error()
    torch.cuda.synchronize()
    return kout.cpu().numpy(), vout.cpu().numpy()


def test_noalloc_sort_matches_allocating_sort_twice_in_a_row():
    assert torch.cuda.is_available()
    dev = torch.device("cuda:0")
    cases = [(MAX_PAIRS, 0, 45, 1000), (300_001, 3, 40, None)]   # two calls, different sizes and bits
    for seed, (n, b0, b1, distinct) in enumerate(cases):
        rng = np.random.default_rng(100 + seed)
        if distinct:
            keys = rng.integers(0, distinct, size=n, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15)
        else:
            keys = rng.integers(0, 2 ** 63, size=n, dtype=np.uint64)
        vals = rng.permutation(n).astype(np.uint32)
        kin = torch.from_numpy(keys.view(np.int64)).to(dev)
        vin = torch.from_numpy(vals.view(np.int32)).to(dev)
        k_ref, v_ref = _sort("tigas_sort_pairs_u64", kin, vin, n, b0, b1)
        k_new, v_new = _sort("tigas_sort_pairs_u64_noalloc", kin, vin, n, b0, b1)
        # integer outputs: bit-exact (the tolerance of every integer parity test)
        assert np.array_equal(k_new, k_ref) and np.array_equal(v_new, v_ref)
        # and both are the stable order of the selected key bits
        sub = (keys >> np.uint64(b0)) & np.uint64((1 << (b1 - b0)) - 1)
        assert np.array_equal(v_new.view(np.uint32), vals[np.argsort(sub, kind="stable")])


def test_noalloc_sort_rejects_sizes_beyond_its_maximum():
    lib = tg.load_library()
    st = lib.tigas_sort_pairs_u64_noalloc(None, None, None, None, ctypes.c_uint64(MAX_PAIRS + 1), 0, 64, None)
    assert st == tb.ERR_INVALID
    assert "1048576" in tg.last_error()
