"""PLY decoding, PLY scene loading and the model registry on the GPU.

Decoding (streamed upload + de-interleaving kernel) must reproduce the
reference PLY reader bit for bit in every format and property type; a scene
loaded from a PLY must render byte-identically to the same arrays loaded
through tigas_scene_load; and the registry must load lazily, share one
resident copy, count references and evict by its (test) clock."""
import threading
import time

import numpy as np
import pytest

import synth
from oracle import ply as oply
from synth import ply as sply

torch = pytest.importorskip("torch")
import paper_2605_08699_b300 as tg  # noqa: E402

pytestmark = pytest.mark.gpu

KEYS = ("means", "log_scales", "quats", "opacity_logits", "sh")


@pytest.fixture(scope="module")
def cuda():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    tg.load_library()
    return torch.device("cuda:0")


def _scene(n, degree=3, seed=3):
    return synth.make_scene(n, synth.BASE_SEED + seed, n_blobs=16, sh_degree=degree)


VARIANTS = [
    dict(fmt="binary_little_endian"),
    dict(fmt="binary_big_endian", shuffle_seed=1, extra_elements=True),
    dict(fmt="ascii", shuffle_seed=2, extra_elements=True),
    dict(fmt="binary_little_endian", shuffle_seed=3, normals=False,
         types={"x": "double", "rot_2": "double", "f_dc_1": "double", "nx": "uchar", "opacity": "short"}),
]


@pytest.mark.parametrize("degree", [0, 3])
@pytest.mark.parametrize("k", range(len(VARIANTS)))
def test_decode_matches_reference_reader(cuda, tmp_path, k, degree):
    n = 3001 if VARIANTS[k]["fmt"] == "ascii" else 70_001   # several chunks of the gather grid, ragged tail
    sc = _scene(n, degree, seed=20 + k)
    path = tmp_path / "s.ply"
    sply.write_ply(path, sc, **VARIANTS[k])
    ref = oply.read_ply(path)
    got = tg.ply_decode(path)
    for key in KEYS:
        np.testing.assert_array_equal(got[key], ref[key], err_msg=key)
    dev = {"means": torch.empty((n, 3), device=cuda), "log_scales": torch.empty((n, 3), device=cuda),
           "quats": torch.empty((n, 4), device=cuda), "opacity_logits": torch.empty((n,), device=cuda),
           "sh": torch.full((n, 16, 3), float("nan"), device=cuda)}
    tg.ply_decode(path, dev)
    for key in KEYS:
        np.testing.assert_array_equal(dev[key].cpu().numpy(), ref[key], err_msg=key)


def test_decode_spans_several_stream_chunks(cuda, tmp_path):
    """A body larger than two 32 MiB staging buffers (the double-buffered
    stream reuses each buffer)."""
    n = 300_000   # 62 floats per record: 74 MB
    sc = _scene(n, 3, seed=31)
    path = tmp_path / "big.ply"
    sply.write_ply(path, sc)
    got = tg.ply_decode(path)
    ref = oply.read_ply(path)
    for key in KEYS:
        np.testing.assert_array_equal(got[key], ref[key], err_msg=key)


@pytest.mark.parametrize("storage", [tg.STORAGE_FP32, tg.STORAGE_FP16])
@pytest.mark.parametrize("degree", [0, 1, 3])
def test_ply_scene_renders_like_the_same_arrays(cuda, tmp_path, storage, degree):
    sc = _scene(40_000, degree, seed=40 + degree)
    path = tmp_path / "m.ply"
    sply.write_ply(path, sc, fmt="binary_little_endian", shuffle_seed=7)
    ref = oply.read_ply(path)
    pose = synth.config_trajectory(2)[10]
    w, h = 333, 197
    K = synth.default_intrinsics(w, h)
    with tg.scene_load_ply(path, storage, background=(0.1, 0.2, 0.3)) as a, \
            tg.scene_load(ref["means"], ref["log_scales"], ref["quats"], ref["opacity_logits"], ref["sh"],
                          ref["sh_degree"], storage, background=(0.1, 0.2, 0.3)) as b:
        assert a.bytes == b.bytes
        fa, fb = tg.render(a, pose, K, w, h), tg.render(b, pose, K, w, h)
    assert fa.any() and np.array_equal(fa, fb)


def test_load_errors_are_reported(cuda, tmp_path):
    with pytest.raises(tg.TigasError) as e:
        tg.scene_load_ply(tmp_path / "absent.ply")
    assert e.value.status == tg.ERR_IO
    p = tmp_path / "bad.ply"
    p.write_bytes(b"ply\nformat ascii 1.0\nelement vertex 1\nproperty float x\nend_header\n1\n")
    with pytest.raises(tg.TigasError) as e:
        tg.scene_load_ply(p)
    assert e.value.status == tg.ERR_INVALID
    p2 = tmp_path / "short.ply"   # ascii body with too few values
    sply.write_ply(p2, _scene(4, 0), fmt="ascii")
    txt = p2.read_bytes()
    p2.write_bytes(txt[:txt.rindex(b" ")] + b"\n")
    with pytest.raises(tg.TigasError) as e:
        tg.scene_load_ply(p2)
    assert e.value.status == tg.ERR_INVALID


def test_launch_sets_of_a_freed_scene_are_never_reused(cuda):
    """Captured launch sets hold a scene's device pointers.  Scenes freed and
    loaded in turn (a new scene may reuse a freed one's host address) must each
    render their own frames: repeated renders (graph replays from the third on)
    equal the scene's direct full-list frame."""
    w, h = 96, 64
    K = synth.default_intrinsics(w, h)
    scenes = [_scene(20_000, 0, seed=61), _scene(35_000, 3, seed=62)]
    for _ in range(3):
        for sc in scenes:
            with tg.scene_from(sc, storage=tg.STORAGE_FP16) as hd:
                want = np.zeros((h, w, 4), np.uint8)
                tg.render_ex(hd, synth.BASE_POSE, K, w, h, out_rgba8=want, sort_mode=tg.SORT_DEPTH_FIRST)
                assert want.any()
                for _ in range(4):
                    assert np.array_equal(tg.render(hd, synth.BASE_POSE, K, w, h), want)


# ------------------------------------------------------------------ registry


@pytest.fixture()
def models(tmp_path):
    sply.write_ply(tmp_path / "alpha.ply", _scene(30_000, 3, seed=51))
    (tmp_path / "beta").mkdir()
    sply.write_ply(tmp_path / "beta" / "beta.ply", _scene(50_000, 0, seed=52))
    return tmp_path


def _frame(scene):
    w, h = 160, 96
    return tg.render(scene, synth.BASE_POSE, synth.default_intrinsics(w, h), w, h)


def test_registry_lazy_shared_refcounted_evicted(cuda, models):
    with tg.Registry(models, storage=tg.STORAGE_FP16, idle_timeout_s=10.0) as reg:
        reg.set_clock(100.0)
        assert not reg.model("alpha")["loaded"]
        a1 = reg.acquire("alpha")
        m = reg.model("alpha")
        assert m["loaded"] and m["users"] == 1 and m["loads"] == 1 and m["resident_bytes"] > 0
        assert not reg.model("beta")["loaded"]   # only what was asked for
        a2 = reg.acquire("alpha")                 # a second client shares the resident copy
        assert a2.handle == a1.handle and reg.model("alpha")["loads"] == 1 and reg.model("alpha")["users"] == 2
        with tg.scene_load_ply(reg.model("alpha")["ply_path"], tg.STORAGE_FP16) as direct:
            assert np.array_equal(_frame(a1), _frame(direct))
        reg.set_clock(200.0)
        assert reg.evict_idle() == 0              # in use: never evicted
        a1.free()
        reg.set_clock(205.0)
        a2.free()                                 # last use at t = 205
        assert reg.model("alpha")["idle_seconds"] == 0.0
        reg.set_clock(214.9)
        assert reg.evict_idle() == 0 and reg.model("alpha")["loaded"]
        assert abs(reg.model("alpha")["idle_seconds"] - 9.9) < 1e-9
        reg.set_clock(215.0)
        assert reg.evict_idle() == 1
        m = reg.model("alpha")
        assert not m["loaded"] and m["resident_bytes"] == 0
        a3 = reg.acquire("alpha")                 # loaded again on demand
        assert reg.model("alpha")["loads"] == 2
        assert _frame(a3).any()
        release = tg.load_library().tigas_registry_release
        with tg.scene_load_ply(reg.model("beta")["ply_path"]) as other:
            assert release(reg.handle, other.handle) == tg.ERR_INVALID   # not from this registry
        h = a3.handle
        a3.free()
        assert release(reg.handle, h) == tg.ERR_INVALID                 # returned twice


def test_registry_close_keeps_acquired_scenes(cuda, models):
    reg = tg.Registry(models, idle_timeout_s=0.0)
    s = reg.acquire("beta")
    before = _frame(s)
    reg.close()
    assert np.array_equal(_frame(s), before)   # still resident after the registry is gone
    s.free()


def test_registry_budget_evicts_least_recently_used(cuda, models):
    with tg.Registry(models, storage=tg.STORAGE_FP32, idle_timeout_s=1e9) as probe:
        a = probe.acquire("alpha")
        b = probe.acquire("beta")
        size_a, size_b = probe.model("alpha")["resident_bytes"], probe.model("beta")["resident_bytes"]
        a.free()
        b.free()
    with tg.Registry(models, storage=tg.STORAGE_FP32, idle_timeout_s=1e9,
                     resident_budget_bytes=max(size_a, size_b) + 1024) as reg:
        reg.set_clock(1.0)
        a = reg.acquire("alpha")
        a.free()
        reg.set_clock(2.0)
        b = reg.acquire("beta")                  # alpha is idle: evicted to make room
        assert not reg.model("alpha")["loaded"] and reg.model("beta")["loaded"]
        with pytest.raises(tg.TigasError) as e:  # beta is in use: alpha cannot fit
            reg.acquire("alpha")
        assert e.value.status == tg.ERR_OOM
        b.free()
        a = reg.acquire("alpha")
        assert not reg.model("beta")["loaded"] and reg.model("alpha")["loads"] == 2
        a.free()


def test_registry_background_eviction(cuda, models):
    with tg.Registry(models, idle_timeout_s=0.2) as reg:
        reg.start_eviction(0.05)
        s = reg.acquire("alpha")
        time.sleep(0.5)
        assert reg.model("alpha")["loaded"]      # in use
        s.free()
        t0 = time.time()
        while reg.model("alpha")["loaded"] and time.time() - t0 < 10.0:
            time.sleep(0.05)
        assert not reg.model("alpha")["loaded"]


def test_registry_concurrent_first_acquires_load_once(cuda, models):
    with tg.Registry(models, idle_timeout_s=60.0) as reg:
        got, errs = [], []

        def worker():
            try:
                got.append(reg.acquire("beta"))
            except Exception as e:   # noqa: BLE001
                errs.append(e)

        ts = [threading.Thread(target=worker) for _ in range(8)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        assert not errs
        assert len({s.handle for s in got}) == 1
        m = reg.model("beta")
        assert m["loads"] == 1 and m["users"] == 8
        for s in got:
            s.free()
        assert reg.model("beta")["users"] == 0


def test_registry_scene_serves_through_the_server(cuda, models):
    """A registry scene submitted to the server stays valid while the request
    is queued even if the caller returns it and the model is evicted."""
    with tg.Registry(models, idle_timeout_s=0.0) as reg:
        reg.set_clock(1.0)
        s = reg.acquire("alpha")
        ref = _frame(s)
        with tg.Server(max_batch=1, max_inflight=1) as srv:
            out = np.zeros((96, 160, 4), np.uint8)
            srv.submit(s, synth.BASE_POSE, synth.default_intrinsics(160, 96), 160, 96, out, client_id=1)
            s.free()
            reg.set_clock(2.0)
            reg.evict_idle()
            done = []
            t0 = time.time()
            while not done and time.time() - t0 < 30.0:
                done += srv.poll(16, timeout_us=2_000_000)
            assert [c.status for c in done] == [tg.OK]
            assert np.array_equal(out, ref)
