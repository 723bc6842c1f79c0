"""The C-ABI library loads and exports every declared symbol (no GPU needed),
and argument validation rejects bad input before any CUDA work."""
import ctypes
import math
import os
import re
import subprocess

import numpy as np
import pytest

import paper_2605_08699_b300 as tg
from paper_2605_08699_b300 import tigas as tb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tigas.h")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(tb.LIB_PATH):
        from paper_2605_08699_b300 import build
        build.build()
    return tg.load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tigas_[a-z0-9_]+)\s*\(", text)))


def test_header_declarations_match_binding():
    assert declared_functions() == sorted(tb.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.check_output(["nm", "-D", "--defined-only", tb.LIB_PATH], text=True)
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    for name in declared_functions():
        assert name in exported, name
        assert getattr(lib, name) is not None
    # nothing but the C ABI is exported
    assert {e for e in exported if not e.startswith("tigas_")} <= {"_init", "_fini"}


def test_version_and_counters(lib):
    assert "sm_103a" in tg.version()
    assert tg.kernel_launches() >= 0


def _status(name, *args):
    return getattr(tg.load_library(), name)(*args)


def test_invalid_arguments_rejected_without_gpu(lib):
    pose = tb.Pose(0.0, 0.0, (ctypes.c_double * 3)(0, 0, -3))
    k = tb.Intrinsics(100, 100, 50, 50)
    buf = np.zeros(16, np.uint8)
    assert _status("tigas_render", None, ctypes.byref(pose), ctypes.byref(k), 2, 2, buf.ctypes.data) == tb.ERR_INVALID
    assert "scene" in tg.last_error()
    assert _status("tigas_scene_load", None, None) == tb.ERR_INVALID
    d = tb.SceneDesc(0, 3, 0, None, None, None, None, None, 0, (ctypes.c_float * 3)(0, 0, 0))
    h = ctypes.c_void_p()
    assert _status("tigas_scene_load", ctypes.byref(d), ctypes.byref(h)) == tb.ERR_INVALID
    d.n, d.sh_degree = 10, 4
    assert _status("tigas_scene_load", ctypes.byref(d), ctypes.byref(h)) == tb.ERR_INVALID
    assert "sh_degree" in tg.last_error()
    d.sh_degree, d.storage = 3, 7
    assert _status("tigas_scene_load", ctypes.byref(d), ctypes.byref(h)) == tb.ERR_INVALID
    assert _status("tigas_scene_free", None) == tb.ERR_INVALID
    assert _status("tigas_sort_pairs_u64", None, None, None, None, 5, 0, 64, None) == tb.ERR_INVALID
    assert _status("tigas_sort_pairs_u64", None, None, None, None, 0, 10, 5, None) == tb.ERR_INVALID
    cfg = tb.ServerConfig(0, 65, 1, 0)
    s = ctypes.c_void_p()
    assert _status("tigas_server_create", ctypes.byref(cfg), ctypes.byref(s)) == tb.ERR_INVALID
    n = ctypes.c_int()
    assert _status("tigas_server_poll", None, None, 0, 0, ctypes.byref(n)) == tb.ERR_INVALID


def test_pose_validation_messages(lib):
    from paper_2605_08699_b300.tigas import _check, TigasError
    k = tb.Intrinsics(100, 100, 50, 50)
    fake_scene = None
    for pose, w, h in [(tb.Pose(math.nan, 0, (ctypes.c_double * 3)(0, 0, 0)), 4, 4),
                       (tb.Pose(0, 0, (ctypes.c_double * 3)(0, math.inf, 0)), 4, 4)]:
        st = _status("tigas_render_ex", fake_scene, ctypes.byref(pose), ctypes.byref(k), w, h, None, None, None, 0, None)
        assert st == tb.ERR_INVALID
    with pytest.raises(TigasError):
        _check(tb.ERR_INVALID)


def test_schedule_set_get_and_range_checks():
    tg.load_library()
    before = tg.get_schedules()
    try:
        tg.set_schedule(12, 256, 3, 16, 4)
        for n in range(1, 65):   # every class
            assert tg.get_schedule(n) == {"n_slices": 12, "first_slice_inv": 256, "blend_ctas_per_sm": 3,
                                          "blend_batch": 16, "views_per_set": 4}
        tg.set_schedule(12, 256, 3, 0, 0)   # blend batch 0 is read as 32
        assert tg.get_schedule(8)["blend_batch"] == 32
        for bad in [(0, 64, 0), (17, 64, 0), (8, 0, 0), (8, 5000, 0), (8, 64, -1), (8, 64, 65), (8, 64, 0, 8),
                    (8, 64, 0, 64), (8, 64, 0, 32, -1), (8, 64, 0, 32, 65)]:
            for n_views in (0, 5):
                with pytest.raises(tg.TigasError) as e:
                    tg.set_schedule(*bad, n_views=n_views)
                assert e.value.status == tg.ERR_INVALID
        assert tg.get_schedule(5)["n_slices"] == 12   # a rejected call changes nothing
        for n in (0, 65):
            with pytest.raises(tg.TigasError):
                tg.get_schedule(n)
            if n:
                with pytest.raises(tg.TigasError):
                    tg.set_schedule(4, 16, n_views=n)
    finally:
        tg.set_schedules(before)


def test_schedule_classes_are_1_2_3to4_5to8_and_so_on():
    tg.load_library()
    before = tg.get_schedules()
    try:
        tg.set_schedule(6, 64)
        tg.set_schedule(2, 8, n_views=3)   # the class of 3 and 4 views only
        got = {n: tg.get_schedule(n)["n_slices"] for n in range(1, 65)}
        assert got == {n: 2 if n in (3, 4) else 6 for n in range(1, 65)}
        tg.set_schedule(5, 32, n_views=40)   # 33..64
        assert [tg.get_schedule(n)["n_slices"] for n in (32, 33, 64)] == [6, 5, 5]
        tg.set_schedule(1, 1, n_views=1)
        assert [tg.get_schedule(n)["n_slices"] for n in (1, 2)] == [1, 6]
    finally:
        tg.set_schedules(before)


def test_default_schedules_take_fewer_slices_for_smaller_launch_sets():
    # a fresh process has the defaults
    import subprocess
    import sys
    code = ("import paper_2605_08699_b300 as tg; tg.load_library(); "
            "print(tg.get_schedule(1)['n_slices'], tg.get_schedule(1)['first_slice_inv'], "
            "*[tg.get_schedule(n)['n_slices'] for n in (2, 3, 4, 5, 8, 64)])")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, check=True,
                         cwd=root).stdout.split()
    assert [int(x) for x in out] == [3, 16, 4, 5, 5, 6, 6, 6]


def test_profile_stage_mask_checks(lib):
    assert _status("tigas_profile_stages", ctypes.c_uint32(1 << 7)) == tb.ERR_INVALID
    assert _status("tigas_profile_stages", ctypes.c_uint32(0xFFFFFFFF)) == tb.ERR_INVALID
    tg.profile_stages(["blend", "preprocess"])
    tg.profile_stages([])
    tg.profile_enable(False)
    with pytest.raises(ValueError):
        tg.profile_stages(["no_such_stage"])


def test_async_and_quality_arguments_rejected_without_gpu(lib):
    pose = tb.Pose(0.0, 0.0, (ctypes.c_double * 3)(0, 0, -3))
    k = tb.Intrinsics(100, 100, 50, 50)
    w = (ctypes.c_int * 1)(4)
    t = ctypes.c_void_p()
    outs = (ctypes.c_void_p * 1)(None)
    # null scene, null ticket output, null output buffer, n_views out of range, null ticket
    assert _status("tigas_render_batch_async", None, 1, ctypes.byref(pose), ctypes.byref(k), w, w, outs, None,
                   ctypes.byref(t)) == tb.ERR_INVALID
    assert _status("tigas_render_batch_async", None, 1, ctypes.byref(pose), ctypes.byref(k), w, w, outs, None,
                   None) == tb.ERR_INVALID
    assert _status("tigas_render_batch_async", ctypes.c_void_p(1), 0, ctypes.byref(pose), ctypes.byref(k), w, w,
                   outs, None, ctypes.byref(t)) == tb.ERR_INVALID
    assert _status("tigas_render_batch_async", ctypes.c_void_p(1), 1, ctypes.byref(pose), ctypes.byref(k), w, w,
                   outs, None, ctypes.byref(t)) == tb.ERR_INVALID
    assert _status("tigas_render_wait", None) == tb.ERR_INVALID
    assert _status("tigas_ply_probe", None, None) == tb.ERR_INVALID
    assert _status("tigas_ply_decode", None, None, None, None, None, None, 0) == tb.ERR_INVALID
    assert _status("tigas_scene_load_ply", None, 0, None, None) == tb.ERR_INVALID
    for name in ("tigas_registry_scan", "tigas_registry_evict_idle"):
        assert _status(name, None, None, None) == tb.ERR_INVALID if name == "tigas_registry_scan" else \
            _status(name, None, None) == tb.ERR_INVALID
    assert _status("tigas_registry_close", None) == tb.ERR_INVALID
    assert _status("tigas_registry_set_clock", None, ctypes.c_double(1.0)) == tb.ERR_INVALID


def test_fault_injection_and_workspace_arguments_without_gpu(lib):
    # the injection knob is host state: it validates and arms without any CUDA call
    assert _status("tigas_debug_fail_alloc", 2, ctypes.c_int64(1), ctypes.c_int64(1)) == tb.ERR_INVALID
    assert _status("tigas_debug_fail_alloc", 0, ctypes.c_int64(-1), ctypes.c_int64(1)) == tb.ERR_INVALID
    assert _status("tigas_debug_fail_alloc", 1, ctypes.c_int64(3), ctypes.c_int64(0)) == tb.ERR_INVALID
    assert _status("tigas_debug_fail_alloc", 0, ctypes.c_int64(2), ctypes.c_int64(5)) == tb.OK
    assert _status("tigas_debug_fail_alloc", 0, ctypes.c_int64(0), ctypes.c_int64(0)) == tb.OK   # cleared
    # with no render context created yet there is nothing to free
    assert _status("tigas_release_workspace") == tb.OK
