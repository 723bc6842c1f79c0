"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Workload 1 (100k Gaussians in 8 isotropic blobs, 320x240, 300 tiles) is
compared in full: per-Gaussian decisions, every tile list, ranges, colour.
Ragged sizes, empty frames, degenerate scenes and both sort modes are
covered; the full-size 3M / 1080p workload is compared on sampled tiles and
pixels in the configuration the benchmark times.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth
from tests import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2605_08699_b300 as tg  # noqa: E402


def _diag(name, obj):
    d = os.environ.get("TIGAS_DIAG_DIR")   # optional folder for per-test diagnostics
    if d and os.path.isdir(d):
        with open(os.path.join(d, "parity_diag.jsonl"), "a") as f:
            f.write(json.dumps({"test": name, **obj}) + "\n")


@pytest.fixture(scope="module")
def cuda():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    tg.load_library()
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def s1():
    return synth.config_scene(1)


@pytest.fixture(scope="module")
def h1(cuda, s1):
    h = tg.scene_from(s1)
    yield h
    h.free()


K1 = synth.default_intrinsics(320, 240)


# ------------------------------------------------------------------ sort


@pytest.mark.parametrize("n,bits,distinct", [(1, (0, 64), None), (4095, (0, 64), None), (4096, (0, 40), None),
                                             (4097, (5, 37), None), (100_003, (0, 64), None),
                                             (1_000_000, (0, 45), 97), (2_500_000, (32, 45), 300)])
def test_radix_sort_matches_stable_sort(cuda, n, bits, distinct):
    rng = np.random.default_rng(n)
    if distinct:
        keys = rng.integers(0, distinct, size=n, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15)
    else:
        keys = rng.integers(0, 2 ** 63, size=n, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, size=n, dtype=np.uint64)
    vals = np.arange(n, dtype=np.uint32)
    b0, b1 = bits
    mask = np.uint64((1 << (b1 - b0)) - 1) if b1 - b0 < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
    sub = (keys >> np.uint64(b0)) & mask
    order = np.argsort(sub, kind="stable")
    kin = torch.from_numpy(keys.view(np.int64)).to(cuda)
    vin = torch.from_numpy(vals.view(np.int32)).to(cuda)
    kout, vout = torch.empty_like(kin), torch.empty_like(vin)
    tg.sort_pairs_u64(kin, vin, kout, vout, n, b0, b1)
    assert np.array_equal(vout.cpu().numpy().view(np.uint32), vals[order])
    assert np.array_equal(kout.cpu().numpy().view(np.uint64), keys[order])
    assert np.array_equal(kin.cpu().numpy().view(np.uint64), keys)   # input untouched


# ---------------------------------------------------------- integer work


@pytest.mark.parametrize("mode", [tg.SORT_DEPTH_FIRST, tg.SORT_FULL64])
def test_workload1_integer_parity(h1, s1, mode):
    dbg = tg.debug_render(h1, synth.BASE_POSE, K1, 320, 240, sort_mode=mode)
    pr = oracle.preprocess(s1, synth.BASE_POSE, K1, 320, 240)
    g = parity.check_per_gaussian(dbg, pr)
    t = parity.check_tile_lists(dbg, pr)
    # diagnostics that size the guard bands: FP32 vs FP64 decision quantities
    v = (pr.visible > 0) & (dbg["visible"] > 0)
    q_rel = np.abs(dbg["q"][v] - pr.dq[v, 2]) / pr.dq[v, 2]
    u_abs = np.abs(dbg["uv"][v, 0] - pr.uvz[v, 0])
    z_rel = np.abs(dbg["depth"][v] - pr.uvz[v, 2]) / pr.uvz[v, 2]
    _diag("workload1_integer", {"mode": mode, **g, **t, "pairs": dbg["pairs"],
                                "q_rel_max": float(q_rel.max()), "u_abs_max": float(u_abs.max()),
                                "z_rel_max": float(z_rel.max())})
    assert g["ambiguous"] < 0.002 * s1.n
    assert dbg["pairs"] == int(pr.tiles_touched[dbg["visible"] > 0].sum()) or g["ambiguous_flipped"] > 0
    # FP32 decision quantities sit inside the guard bands
    assert q_rel.max() < oracle.DEFAULT_GUARDS[2]
    scale = np.abs(pr.uvz[v, 0] - K1.cx) + K1.cx + pr.radius[v] + 1.0
    assert np.all(u_abs < oracle.DEFAULT_GUARDS[3] * scale)
    assert z_rel.max() < 2.0 ** -20


def test_workload1_ranges_exact_when_no_flip(h1, s1):
    dbg = tg.debug_render(h1, synth.BASE_POSE, K1, 320, 240)
    pr = oracle.preprocess(s1, synth.BASE_POSE, K1, 320, 240)
    g = parity.check_per_gaussian(dbg, pr)
    orr, ov = oracle.tile_lists(pr)
    gr = dbg["ranges"].astype(np.int64)
    gv = dbg["values"].astype(np.int64)
    # every path: the ranges are contiguous in tile order and cover the pair array ...
    assert gr[0, 0] == 0 and np.array_equal(gr[1:, 0], gr[:-1, 1]) and gr[-1, 1] == dbg["pairs"]
    # ... each tile's unambiguous entries are exactly as many as the oracle's, and a
    # tile with no ambiguous member in either list has exactly the oracle's length
    amb = pr.amb > 0
    clean = 0
    for t in range(len(orr)):
        g_t, o_t = gv[gr[t, 0]:gr[t, 1]], ov[orr[t, 0]:orr[t, 1]]
        assert np.count_nonzero(~amb[g_t]) == np.count_nonzero(~amb[o_t]), f"tile {t}"
        if not amb[g_t].any() and not amb[o_t].any():
            assert g_t.size == o_t.size, f"tile {t}"
            clean += 1
    assert clean > 0   # (181 of the 300 tiles hold no ambiguous Gaussian on this seed)
    # ... and without a flipped decision the ranges equal the oracle's exactly
    if g["ambiguous_flipped"] == 0:
        assert np.array_equal(gr, orr)
    _diag("workload1_ranges", {**g, "clean_tiles": clean, "tiles": len(orr)})


def test_support_rule_scene_on_gpu(cuda):
    # a Gaussian whose alpha >= 1/255 region reaches past its 3-sigma rectangle:
    # every schedule must leave the pixels outside the rectangle at the background
    from tests.test_oracle_raster import support_rule_scene
    sc, K, W, H = support_rule_scene()
    pr = oracle.preprocess(sc, synth.BASE_POSE, K, W, H)
    ref = oracle.render(pr)
    with tg.scene_from(sc) as h:
        for mode in (tg.SORT_DEPTH_FIRST, tg.SORT_FULL64):
            dbg = tg.debug_render(h, synth.BASE_POSE, K, W, H, sort_mode=mode)
            assert tuple(dbg["rect"][0]) == (1, 0, 3, 2) and dbg["radius"][0] == 15
            f = dbg["rgba_f32"]
            assert np.all(f[:, 48:] == 0.0)
            assert np.max(np.abs(f.astype(np.float64) - ref)) < 2e-5
        fast = np.zeros((H, W, 4), np.float32)
        tg.render_ex(h, synth.BASE_POSE, K, W, H, out_rgba_f32=fast, sort_mode=tg.SORT_SLICED)
        assert np.array_equal(fast, f)


def test_sort_modes_give_identical_frames(h1):
    pose = synth.Pose(0.3, -0.2, (0.1, 0.05, -2.8))
    a = tg.debug_render(h1, pose, K1, 320, 240, sort_mode=tg.SORT_DEPTH_FIRST)
    b = tg.debug_render(h1, pose, K1, 320, 240, sort_mode=tg.SORT_FULL64)
    assert a["pairs"] == b["pairs"]
    assert np.array_equal(a["values"], b["values"]) and np.array_equal(a["ranges"], b["ranges"])
    assert np.array_equal(a["rgba_f32"], b["rgba_f32"])


# ------------------------------------------------- sliced schedule = full


@pytest.mark.parametrize("k,w,h", [(0, 320, 240), (150, 320, 240), (299, 97, 61), (40, 1000, 3)])
def test_sliced_schedule_gives_the_full_list_frame(h1, s1, k, w, h):
    pose = synth.config_trajectory(1)[k]
    K = synth.default_intrinsics(w, h)
    full = tg.debug_render(h1, pose, K, w, h, sort_mode=tg.SORT_DEPTH_FIRST)
    sliced = tg.debug_render(h1, pose, K, w, h, sort_mode=tg.SORT_SLICED)
    assert np.array_equal(full["rgba_f32"], sliced["rgba_f32"])
    assert np.array_equal(full["visible"], sliced["visible"]) and np.array_equal(full["rect"], sliced["rect"])
    assert sliced["pairs"] <= full["pairs"]
    parity.assert_colour(sliced["rgba_f32"], oracle.render(oracle.preprocess(s1, pose, K, w, h)))


@pytest.mark.parametrize("k,w,h", [(0, 320, 240), (150, 320, 240), (299, 97, 61), (40, 1000, 3), (75, 640, 360)])
def test_sliced_fast_path_gives_the_full_list_frame(h1, k, w, h):
    # the render path (no debug outputs) cuts every rectangle to the tiles its
    # alpha >= 1/255 region can reach: the frame must not change by one bit
    pose = synth.config_trajectory(1)[k]
    K = synth.default_intrinsics(w, h)
    full = tg.debug_render(h1, pose, K, w, h, sort_mode=tg.SORT_DEPTH_FIRST)
    fast = np.zeros((h, w, 4), np.float32)
    st = tg.render_ex(h1, pose, K, w, h, out_rgba_f32=fast, sort_mode=tg.SORT_SLICED)
    assert np.array_equal(full["rgba_f32"], fast)
    assert st["n_pairs"] <= full["pairs"]


def test_sliced_debug_render_has_no_whole_lists(h1):
    with pytest.raises(tg.TigasError):
        tg.load_library()
        from paper_2605_08699_b300 import tigas as tb
        import ctypes
        d = tb.DebugFrame(None, None, None, None, None, None, 1, 4, 1, None)
        pairs = ctypes.c_uint64()
        tb._check(tg.load_library().tigas_debug_render(h1.handle, ctypes.byref(tb.make_pose(synth.BASE_POSE)),
                                                       ctypes.byref(tb.make_intrinsics(K1)), 320, 240,
                                                       tg.SORT_SLICED, ctypes.byref(d), ctypes.byref(pairs)))


# ---------------------------------------------------------------- colour


def test_workload1_colour_parity(h1, s1):
    dbg = tg.debug_render(h1, synth.BASE_POSE, K1, 320, 240)
    ref = oracle.render(oracle.preprocess(s1, synth.BASE_POSE, K1, 320, 240))
    st = parity.assert_colour(dbg["rgba_f32"], ref)
    _diag("workload1_colour", st)


def test_rgba8_is_rounded_float_output(h1, cuda):
    out8 = torch.empty((240, 320, 4), dtype=torch.uint8, device=cuda)
    out32 = torch.empty((240, 320, 4), dtype=torch.float32, device=cuda)
    tg.render_ex(h1, synth.BASE_POSE, K1, 320, 240, out_rgba8=out8, out_rgba_f32=out32)
    f = out32.cpu().numpy().astype(np.float64)
    expect = np.floor(np.clip(f, 0, 1) * 255.0 + 0.5)
    got = out8.cpu().numpy().astype(np.float64)
    # FP32 rounding of x*255+0.5 can differ from the FP64 value by one code at exact halves
    assert np.max(np.abs(got - expect)) <= 1 and np.mean(got != expect) < 1e-4
    host = tg.render(h1, synth.BASE_POSE, K1, 320, 240)
    assert np.array_equal(host, out8.cpu().numpy())


@pytest.mark.parametrize("k", [0, 60, 120, 299])
def test_trajectory_poses_colour(h1, s1, k):
    pose = synth.config_trajectory(1)[k]
    dbg = tg.debug_render(h1, pose, K1, 320, 240)
    pr = oracle.preprocess(s1, pose, K1, 320, 240)
    parity.check_per_gaussian(dbg, pr)
    parity.assert_colour(dbg["rgba_f32"], oracle.render(pr))


@pytest.mark.parametrize("w,h", [(1, 1), (17, 33), (250, 7), (321, 241), (1000, 3)])
def test_ragged_sizes(h1, s1, w, h):
    K = synth.default_intrinsics(w, h)
    dbg = tg.debug_render(h1, synth.BASE_POSE, K, w, h)
    pr = oracle.preprocess(s1, synth.BASE_POSE, K, w, h)
    parity.check_per_gaussian(dbg, pr)
    parity.check_tile_lists(dbg, pr)
    parity.assert_colour(dbg["rgba_f32"], oracle.render(pr))


def test_empty_frame_camera_facing_away(h1):
    pose = synth.Pose(math.pi, 0.0, (0.0, 0.0, -3.0))      # looks along -z, away from the scene
    dbg = tg.debug_render(h1, pose, K1, 320, 240)
    assert dbg["pairs"] == 0 and dbg["visible"].sum() == 0
    assert np.all(dbg["rgba_f32"] == 0.0)


def test_zero_opacity_scene_is_background(cuda, s1):
    s = s1.subset(np.arange(5000))
    s.opacity_logits[:] = -30.0
    with tg.scene_from(s, background=(0.25, 0.5, 0.75)) as h:
        img = tg.debug_render(h, synth.BASE_POSE, K1, 320, 240)["rgba_f32"]
    assert np.all(img[..., :3] == np.array([0.25, 0.5, 0.75], np.float32)) and np.all(img[..., 3] == 0)


def test_camera_inside_scene_near_plane(cuda, s1):
    pose = synth.Pose(0.4, 0.1, (0.0, 0.1, 0.0))           # in the middle of the blobs
    with tg.scene_from(s1) as h:
        dbg = tg.debug_render(h, pose, K1, 320, 240)
    pr = oracle.preprocess(s1, pose, K1, 320, 240)
    assert (pr.cull == 1).sum() > 10000
    parity.check_per_gaussian(dbg, pr)
    parity.check_tile_lists(dbg, pr)
    parity.assert_colour(dbg["rgba_f32"], oracle.render(pr))


@pytest.mark.parametrize("deg", [0, 1, 2])
def test_lower_sh_degrees(cuda, s1, deg):
    s = s1.subset(np.arange(30000))
    s.sh_degree = deg
    pose = synth.Pose(0.5, 0.3, (0.2, -0.1, -3.0))
    with tg.scene_from(s) as h:
        dbg = tg.debug_render(h, pose, K1, 320, 240)
    pr = oracle.preprocess(s, pose, K1, 320, 240)
    parity.assert_colour(dbg["rgba_f32"], oracle.render(pr))


def test_fp16_storage_against_fp32_oracle(cuda, s1):
    with tg.scene_from(s1, storage=tg.STORAGE_FP16) as h:
        assert h.bytes == ((s1.n + 31) // 32) * 32 * 128
        dbg = tg.debug_render(h, synth.BASE_POSE, K1, 320, 240)
    ref = oracle.render(oracle.preprocess(s1, synth.BASE_POSE, K1, 320, 240))
    ref16 = oracle.render(oracle.preprocess(s1, synth.BASE_POSE, K1, 320, 240, storage_half=True))
    st = parity.colour_stats(dbg["rgba_f32"], ref)
    st16 = parity.colour_stats(dbg["rgba_f32"], ref16)
    _diag("fp16_workload1", {"vs_fp32_oracle": st, "vs_fp16_oracle": st16})
    assert st["psnr_rgb"] >= 50.0
    assert st16["psnr_rgb"] >= st["psnr_rgb"] - 1.0


# ------------------------------------------------------------ batching


def test_batch_equals_single_renders(h1, cuda):
    levels = [(480, 270), (320, 240), (97, 61), (1280, 720), (768, 432)]
    poses = synth.trajectory(77, 5)
    intrs = [synth.default_intrinsics(w, h) for w, h in levels]
    outs = [torch.empty((h, w, 4), dtype=torch.uint8, device=cuda) for w, h in levels]
    tg.render_batch(h1, poses, intrs, [w for w, _ in levels], [h for _, h in levels], outs)
    for (w, h), p, k, o in zip(levels, poses, intrs, outs):
        single = tg.render(h1, p, k, w, h)
        assert np.array_equal(single, o.cpu().numpy())
    # host outputs through the batch entry point
    houts = [np.zeros((h, w, 4), np.uint8) for w, h in levels]
    tg.render_batch(h1, poses, intrs, [w for w, _ in levels], [h for _, h in levels], houts)
    for ho, o in zip(houts, outs):
        assert np.array_equal(ho, o.cpu().numpy())


# ----------------------------------------------------------- CUDA graphs


def _batch(h, poses, levels, cuda):
    intrs = [synth.default_intrinsics(w, hh) for w, hh in levels]
    outs = [torch.empty((hh, w, 4), dtype=torch.uint8, device=cuda) for w, hh in levels]
    tg.render_batch(h, poses, intrs, [w for w, _ in levels], [hh for _, hh in levels], outs)
    return [o.cpu().numpy() for o in outs]


def test_wide_and_compact_rectangles_give_the_same_frames(h1, cuda):
    """Launch sets whose views all fit 127 x 127 tiles, with at most 16 views,
    carry compact rectangles (with their entry ids) through the depth sort; a
    wider view or a 17th view switches the whole set to the wide form."""
    levels = [(320, 240), (97, 61)]
    poses = synth.trajectory(91, 3)
    compact = _batch(h1, poses[:2], levels, cuda)
    wide = _batch(h1, poses, levels + [(2100, 40)], cuda)
    for a, b in zip(compact, wide[:2]):
        assert np.array_equal(a, b)
    p17 = synth.trajectory(92, 17)
    many = _batch(h1, p17, [(64, 48)] * 17, cuda)
    for p, o in zip(p17, many):
        assert np.array_equal(tg.render(h1, p, synth.default_intrinsics(64, 48), 64, 48), o)
    # the boundary: 127 tile columns are compact, 128 are not; both match the full lists
    for w in (2032, 2033):
        pose, K = synth.config_trajectory(1)[30], synth.default_intrinsics(w, 40)
        full = tg.debug_render(h1, pose, K, w, 40, sort_mode=tg.SORT_DEPTH_FIRST)
        fast = np.zeros((40, w, 4), np.float32)
        tg.render_ex(h1, pose, K, w, 40, out_rgba_f32=fast, sort_mode=tg.SORT_SLICED)
        assert np.array_equal(full["rgba_f32"], fast)


def test_launch_set_of_more_than_65536_tiles(h1, cuda):
    """Nine 1080p views hold 73440 tiles: tile ids of 17 bits, so the pair sort
    runs three passes and each run of 256 tiles of the tile ranges is found by
    search rather than from the second pass's digit bases.  Every frame equals
    its single-view render (8160 tiles: the digit-bases path)."""
    poses = synth.trajectory(93, 9)
    many = _batch(h1, poses, [(1920, 1080)] * 9, cuda)
    K = synth.default_intrinsics(1920, 1080)
    for p, o in zip(poses, many):
        assert np.array_equal(tg.render(h1, p, K, 1920, 1080), o)


def test_graph_replay_equals_direct_launches(h1, cuda):
    levels = [(480, 270), (320, 240), (97, 61)]
    tr = synth.trajectory(11, 40)
    tg.set_graphs(False)
    ref = [_batch(h1, tr[i:i + 3], levels, cuda) for i in (0, 10, 20)]
    tg.set_graphs(True)
    # first: direct fixed-capacity launch set; second: exact + capture; third: replay
    got = [_batch(h1, tr[i:i + 3], levels, cuda) for i in (0, 10, 20)]
    for a, b in zip(ref, got):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


def test_graph_overflow_falls_back_to_exact(cuda, s1):
    # capture on a far pose (few pairs), replay on a near one (far more pairs than
    # the captured capacity): the frame must still be right
    levels = [(320, 240)]
    far = [synth.Pose(0.0, 0.0, (0.0, 0.0, -12.0))]
    near = [synth.Pose(0.1, 0.05, (0.0, 0.0, -2.2))]
    with tg.scene_from(s1) as h:
        tg.set_graphs(False)
        ref = _batch(h, near, levels, cuda)
        tg.set_graphs(True)
        _batch(h, far, levels, cuda)
        _batch(h, far, levels, cuda)
        got = _batch(h, near, levels, cuda)
        got2 = _batch(h, near, levels, cuda)
    assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[0], got2[0])


def test_async_launch_sets_equal_synchronous_ones(cuda, s1):
    """Tickets kept in flight (the next launch set queued before the previous
    one is waited on) give the synchronous frames, also when a replayed launch
    set outgrows its captured capacity (far poses captured, then near ones)."""
    levels = [(320, 240), (160, 120)]
    far = [synth.Pose(0.0, 0.0, (0.0, 0.0, -12.0)), synth.Pose(0.2, 0.0, (0.0, 0.0, -11.0))]
    near = [synth.Pose(0.1, 0.05, (0.0, 0.0, -2.2)), synth.Pose(-0.1, 0.0, (0.1, 0.0, -2.4))]
    seq = [far, far, far, near, near, far, near] + [list(synth.trajectory(95 + k, 2)) for k in range(6)]
    intrs = [synth.default_intrinsics(w, h) for w, h in levels]
    with tg.scene_from(s1) as h:
        tg.set_graphs(False)
        want = [_batch(h, poses, levels, cuda) for poses in seq]
        tg.set_graphs(True)
        bufs = [[torch.empty((hh, w, 4), dtype=torch.uint8, device=cuda) for w, hh in levels] for _ in range(2)]
        stream = torch.cuda.Stream()
        got = []
        prev = None
        for k, poses in enumerate(seq):
            t = tg.render_batch_async(h, poses, intrs, [w for w, _ in levels], [hh for _, hh in levels],
                                      bufs[k % 2], stream=stream)
            if prev is not None:
                prev[0].wait()
                got.append([o.cpu().numpy() for o in prev[1]])
            prev = (t, bufs[k % 2])
        prev[0].wait()
        got.append([o.cpu().numpy() for o in prev[1]])
        # pinned host outputs: copied back on the ticket's copy stream
        hosts = [[torch.empty((hh, w, 4), dtype=torch.uint8).pin_memory() for w, hh in levels] for _ in range(2)]
        tk = [tg.render_batch_async(h, seq[k], intrs, [w for w, _ in levels], [hh for _, hh in levels], hosts[i],
                                    stream=stream) for i, k in enumerate((3, 4))]
        for t in tk:
            t.wait()
        for k, hb in zip((3, 4), hosts):
            for a, b in zip(want[k], hb):
                assert np.array_equal(a, b.numpy())
    assert len(got) == len(want)
    for w_set, g_set in zip(want, got):
        for a, b in zip(w_set, g_set):
            assert np.array_equal(a, b)


def test_direct_fixed_capacity_overflow_renders_exactly(cuda, s1):
    # the capacity learned on a far pose is far too small for a new shape on a
    # near pose: the direct launch set overflows and the frame is rendered exactly
    far = [synth.Pose(0.0, 0.0, (0.0, 0.0, -12.0))]
    near = [synth.Pose(0.1, 0.05, (0.0, 0.0, -2.2))]
    with tg.scene_from(s1) as h:
        tg.set_graphs(False)
        ref = _batch(h, near, [(300, 200)], cuda)
        tg.set_graphs(True)   # idle contexts forget learned capacities
        _batch(h, far, [(320, 240)], cuda)
        got = [_batch(h, near, [(300, 200)], cuda) for _ in range(3)]   # direct, exact + capture, replay
    for g in got:
        assert np.array_equal(ref[0], g[0])


# -------------------------------------------------------------- serving


def test_server_results_equal_single_renders(cuda, s1):
    s2 = s1.subset(np.arange(0, 60000))
    with tg.scene_from(s1) as ha, tg.scene_from(s2, storage=tg.STORAGE_FP16) as hb:
        reqs = []
        tr = synth.trajectory(5, 24)
        for i, p in enumerate(tr):
            w, h = synth.ABR_LEVELS[i % 3]
            reqs.append(((ha, hb)[i % 2], p, synth.default_intrinsics(w, h), w, h, i))
        with tg.Server(max_batch=4, max_inflight=2) as srv:
            outs = {}
            for sc, p, k, w, h, c in reqs:
                buf = torch.zeros((h, w, 4), dtype=torch.uint8, device=cuda)
                t = srv.submit(sc, p, k, w, h, buf, client_id=c)
                outs[t] = (buf, sc, p, k, w, h)
            done = []
            while len(done) < len(reqs):
                done += srv.poll(64, timeout_us=2_000_000)
        assert all(c.status == 0 for c in done)
        for c in done:
            buf, sc, p, k, w, h = outs[c.ticket]
            assert c.submit_us <= c.admit_us <= c.done_us
            assert np.array_equal(buf.cpu().numpy(), tg.render(sc, p, k, w, h))


def test_server_latest_pose_wins(cuda, h1):
    with tg.Server(max_batch=1, max_inflight=1) as srv:
        bufs = [np.zeros((240, 320, 4), np.uint8) for _ in range(6)]
        tickets = [srv.submit(h1, synth.BASE_POSE, K1, 320, 240, b, client_id=7) for b in bufs]
        got = {}
        while len(got) < len(tickets):
            for c in srv.poll(16, timeout_us=2_000_000):
                got[c.ticket] = c.status
    # each new request supersedes the queued one of the same client; the last always renders
    assert got[tickets[-1]] == 0
    assert set(got.values()) <= {0, tg.tigas.ERR_AGAIN}
    assert sum(s == tg.tigas.ERR_AGAIN for s in got.values()) >= 1


def test_server_admission_budget_serialises_launch_sets(cuda, h1):
    # a budget below any launch set's workspace admits one request at a time, and
    # only while nothing else is in flight (a lone request is always admitted)
    K = synth.default_intrinsics(160, 120)
    tr = synth.trajectory(23, 8)
    with tg.Server(hbm_budget_bytes=1, max_batch=4, max_inflight=2) as srv:
        bufs = {}
        for i, p in enumerate(tr):
            b = torch.zeros((120, 160, 4), dtype=torch.uint8, device=cuda)
            bufs[srv.submit(h1, p, K, 160, 120, b, client_id=i)] = (b, p)
        done = []
        while len(done) < len(tr):
            done += srv.poll(16, timeout_us=2_000_000)
    assert all(c.status == 0 for c in done)
    spans = sorted((c.admit_us, c.done_us) for c in done)
    assert len(set(spans)) == len(spans)   # one request per launch set
    for (a0, d0), (a1, d1) in zip(spans, spans[1:]):
        assert a1 >= d0                      # no two in flight
    for c in done:
        b, p = bufs[c.ticket]
        assert np.array_equal(b.cpu().numpy(), tg.render(h1, p, K, 160, 120))


def test_server_keeps_a_freed_scene_until_its_requests_finish(cuda, s1):
    K = synth.default_intrinsics(160, 120)
    tr = synth.trajectory(29, 6)
    ref_scene = tg.scene_from(s1)
    try:
        refs = [tg.render(ref_scene, p, K, 160, 120) for p in tr]
        with tg.Server(max_batch=2, max_inflight=1) as srv:
            h = tg.scene_from(s1)
            bufs = {}
            for i, p in enumerate(tr):
                b = torch.zeros((120, 160, 4), dtype=torch.uint8, device=cuda)
                bufs[srv.submit(h, p, K, 160, 120, b, client_id=i)] = (b, i)
            h.free()   # the caller's reference goes; queued requests hold theirs
            done = []
            while len(done) < len(tr):
                done += srv.poll(16, timeout_us=2_000_000)
        assert all(c.status == 0 for c in done)
        for c in done:
            b, i = bufs[c.ticket]
            assert np.array_equal(b.cpu().numpy(), refs[i])
    finally:
        ref_scene.free()


# ------------------------------------------------------- full-size sampled


@pytest.fixture(scope="module")
def s3():
    return synth.config_scene(3)


@pytest.mark.parametrize("storage", [tg.STORAGE_FP16, tg.STORAGE_FP32])
def test_full_size_3m_1080p_sampled(cuda, s3, storage):
    W, H = 1920, 1080
    K = synth.default_intrinsics(W, H)
    pose = synth.config_trajectory(3)[150]
    with tg.scene_from(s3, storage=storage) as h:
        dbg = tg.debug_render(h, pose, K, W, H)
        # the benchmark's launch configuration: the batched entry point
        out = torch.empty((H, W, 4), dtype=torch.uint8, device=cuda)
        tg.render_batch(h, [pose], [K], [W], [H], [out])
    pr = oracle.preprocess(s3, pose, K, W, H, storage_half=storage == tg.STORAGE_FP16)
    # the batched entry point gives the debug render's frame, 8-bit encoded
    f = dbg["rgba_f32"].astype(np.float64)
    got8 = out.cpu().numpy().astype(np.int64)
    assert np.max(np.abs(got8 - np.floor(np.clip(f, 0, 1) * 255 + 0.5))) <= 1
    rng = np.random.default_rng(3)
    TX, TY = pr.tiles_xy
    tiles = [(int(rng.integers(0, TX)), int(rng.integers(0, TY))) for _ in range(12)] + [(TX // 2, TY // 2)]
    if storage == tg.STORAGE_FP32:
        g = parity.check_per_gaussian(dbg, pr)
        t = parity.check_tile_lists(dbg, pr, tiles)
        _diag("full_size_integer", {**g, **t, "pairs": dbg["pairs"]})
    pix = np.stack([rng.integers(0, W, 4000), rng.integers(0, H, 4000)], axis=1).astype(np.int32)
    ref = oracle.render(pr, pixels=pix)
    got = dbg["rgba_f32"][pix[:, 1], pix[:, 0]]
    st = parity.assert_colour(got, ref)
    exp8 = oracle.to_rgba8(ref).astype(np.int64)
    assert np.mean(np.all(np.abs(got8[pix[:, 1], pix[:, 0]] - exp8) <= 1, axis=1)) >= 0.999
    extra = {}
    if storage == tg.STORAGE_FP16:
        # headline error: against the oracle on the original FP32 attributes
        ref32 = oracle.render(oracle.preprocess(s3, pose, K, W, H), pixels=pix)
        extra = {"vs_fp32_oracle": parity.colour_stats(got, ref32)}
        assert extra["vs_fp32_oracle"]["psnr_rgb"] >= 50.0
    _diag("full_size_colour", {"storage": storage, **st, "pairs": dbg["pairs"], **extra})


@pytest.mark.parametrize("storage", [tg.STORAGE_FP32, tg.STORAGE_FP16])
def test_full_size_default_schedule_is_bit_identical_to_whole_lists(cuda, s3, storage):
    """3M Gaussians at 1920x1080: the render path (sliced schedule with
    alpha-cut rectangles: several slices, done tiles, strip items) against the
    whole-list schedule of the debug render, float frames compared bit for bit
    over the whole frame, at two poses."""
    W, H = 1920, 1080
    K = synth.default_intrinsics(W, H)
    tr = synth.config_trajectory(3)
    with tg.scene_from(s3, storage=storage) as h:
        for k in (0, 233):
            full = tg.debug_render(h, tr[k], K, W, H, sort_mode=tg.SORT_DEPTH_FIRST)
            want = full["rgba_f32"].view(np.uint32)
            fast = torch.empty((H, W, 4), dtype=torch.float32, device=cuda)
            # the uninstrumented kernels (no statistics), then the counting ones
            tg.render_ex(h, tr[k], K, W, H, out_rgba_f32=fast, sort_mode=tg.SORT_SLICED, stats=False)
            same = fast.cpu().numpy().view(np.uint32) == want
            st = tg.render_ex(h, tr[k], K, W, H, out_rgba_f32=fast, sort_mode=tg.SORT_SLICED)
            same_counting = fast.cpu().numpy().view(np.uint32) == want
            _diag("full_size_bit_identity", {"storage": storage, "pose": k, "pairs_full": full["pairs"],
                                             "pairs_sliced": st["n_pairs"], "differing": int((~same).sum())})
            assert np.all(same), f"{int((~same).sum())} values differ"
            assert np.all(same_counting), f"{int((~same_counting).sum())} values differ (counting kernels)"
            assert st["n_pairs"] < full["pairs"]


def test_every_launch_path_gives_the_whole_list_frame(cuda):
    """A shape's first render is exact (a host round trip per slice), its
    second exact and captured, its third a graph replay with fixed pair
    capacities, and a new shape after that runs directly with a fixed
    capacity: every float frame equals the whole-list one bit for bit."""
    scene = synth.config_scene(2, n=600_000)
    tr = synth.config_trajectory(2)
    with tg.scene_from(scene, storage=tg.STORAGE_FP16) as h:
        for W, H, k in ((1280, 720, 20), (960, 540, 21)):
            K = synth.default_intrinsics(W, H)
            full = tg.debug_render(h, tr[k], K, W, H, sort_mode=tg.SORT_DEPTH_FIRST)["rgba_f32"].view(np.uint32)
            if W == 1280:
                tg.set_graphs(True)   # idle contexts forget shapes and capacities: the next render is exact
            frames = []
            for _ in range(3):
                f = torch.empty((H, W, 4), dtype=torch.float32, device=cuda)
                tg.render_ex(h, tr[k], K, W, H, out_rgba_f32=f, sort_mode=tg.SORT_SLICED, stats=False)
                frames.append(f.cpu().numpy().view(np.uint32))
            for f in frames:
                assert np.array_equal(f, full)


def test_full_size_8_view_launch_set_view_is_bit_identical(cuda, s3):
    """One view of an 8-view 1080p launch set of the 3M FP16 scene (the timed
    configuration, through tigas_render_batch) against the whole-list debug
    render of the same pose: the launch set's RGBA8 frame equals the kernels'
    8-bit encoding of the debug float frame at every pixel."""
    W, H, V = 1920, 1080, 8
    K = synth.default_intrinsics(W, H)
    poses = [synth.config_trajectory(3, v)[(60 + 11 * v) % 300] for v in range(V)]
    with tg.scene_from(s3, storage=tg.STORAGE_FP16) as h:
        outs = [torch.empty((H, W, 4), dtype=torch.uint8, device=cuda) for _ in range(V)]
        frames = []
        for _ in range(3):   # back to back: first appearance, exact render and capture, graph replay
            tg.render_batch(h, poses, [K] * V, [W] * V, [H] * V, outs)
            torch.cuda.synchronize()
            frames.append({v: outs[v].cpu().numpy() for v in (2, 5)})
        for v in (2, 5):
            full = tg.debug_render(h, poses[v], K, W, H, sort_mode=tg.SORT_DEPTH_FIRST)
            want = parity.encode_rgba8_fp32(full["rgba_f32"])
            for f in frames:
                assert np.array_equal(f[v], want)


def test_full_size_8_view_async_launch_set(cuda, s3):
    """The timed configuration: 8 views of 1080p of the 3M FP16 scene in one
    asynchronous launch set, the next one queued before the wait.  Every
    view equals its own single-view render, and two views meet the colour
    gate against the oracle on sampled pixels."""
    W, H, V = 1920, 1080, 8
    K = synth.default_intrinsics(W, H)
    trajs = [synth.config_trajectory(3, v) for v in range(V)]
    poses = [trajs[v][(40 + 7 * v) % 300] for v in range(V)]
    poses2 = [trajs[v][(41 + 7 * v) % 300] for v in range(V)]
    with tg.scene_from(s3, storage=tg.STORAGE_FP16) as h:
        outs = [torch.empty((H, W, 4), dtype=torch.uint8, device=cuda) for _ in range(V)]
        outs2 = [torch.empty((H, W, 4), dtype=torch.uint8, device=cuda) for _ in range(V)]
        stream = torch.cuda.Stream()
        t1 = tg.render_batch_async(h, poses, [K] * V, [W] * V, [H] * V, outs, stream=stream)
        t2 = tg.render_batch_async(h, poses2, [K] * V, [W] * V, [H] * V, outs2, stream=stream)
        t1.wait()
        t2.wait()
        frames = [o.cpu().numpy() for o in outs]
        for v in (0, 3, 7):
            assert np.array_equal(frames[v], tg.render(h, poses[v], K, W, H))
            assert np.array_equal(outs2[v].cpu().numpy(), tg.render(h, poses2[v], K, W, H))
        f32 = {}
        for v in (0, 5):
            f = np.zeros((H, W, 4), np.float32)
            tg.render_ex(h, poses[v], K, W, H, out_rgba_f32=f)
            f32[v] = f
    rng = np.random.default_rng(11)
    for v in (0, 5):
        pr = oracle.preprocess(s3, poses[v], K, W, H, storage_half=True)
        pix = np.stack([rng.integers(0, W, 3000), rng.integers(0, H, 3000)], axis=1).astype(np.int32)
        ref = oracle.render(pr, pixels=pix)
        st = parity.assert_colour(f32[v][pix[:, 1], pix[:, 0]], ref)
        exp8 = oracle.to_rgba8(ref).astype(np.int64)
        got8 = frames[v][pix[:, 1], pix[:, 0]].astype(np.int64)
        assert np.mean(np.all(np.abs(got8 - exp8) <= 1, axis=1)) >= 0.999
        _diag("full_size_8_view", {"view": v, **st})


# ------------------------------------------------------- failure detection


def test_sort_lookback_wait_times_out_and_device_stays_usable(h1, s1):
    # a look-back wait on counts that nobody publishes gives up and reports
    assert tg.debug_sort_wait_timeout(2048) == tg.ERR_TIMEOUT
    # the context is still usable: a normal frame renders and matches the oracle
    pose = synth.config_trajectory(1)[0]
    w, h = 160, 120
    img = np.zeros((h, w, 4), np.float32)
    tg.render_ex(h1, pose, synth.default_intrinsics(w, h), w, h, out_rgba_f32=img)
    ref = oracle.render(oracle.preprocess(s1, pose, synth.default_intrinsics(w, h), w, h))
    parity.assert_colour(img, ref)
    assert tg.debug_sort_wait_timeout(0) == tg.ERR_INVALID


# ------------------------------------------------------------- scheduling


def test_frames_do_not_depend_on_the_schedule(h1, cuda):
    levels = [(480, 270), (97, 61)]
    tr = synth.trajectory(17, 20)
    base = tg.get_schedules()
    try:
        ref = _batch(h1, tr[3:5], levels, cuda)
        ref1 = tg.render(h1, tr[6], synth.default_intrinsics(480, 270), 480, 270)
        for sch in [(1, 1, 0), (2, 8, 0), (4, 16, 0), (16, 256, 1), (12, 4096, 4), (6, 64, 0, 16), (8, 64, 3, 16)]:
            tg.set_schedule(*sch)
            for _ in range(3):   # direct, exact + capture, replay
                got = _batch(h1, tr[3:5], levels, cuda)
                for a, b in zip(ref, got):
                    assert np.array_equal(a, b), sch
        # one-view launch sets take their own class's schedule
        for sch in [(1, 1, 0), (3, 16, 0), (5, 8, 4, 16)]:
            tg.set_schedule(*sch, n_views=1)
            for _ in range(3):
                assert np.array_equal(tg.render(h1, tr[6], synth.default_intrinsics(480, 270), 480, 270), ref1), sch
    finally:
        tg.set_schedules(base)


def test_server_launch_sets_respect_views_per_set(cuda, h1):
    # the views per launch set of the schedule of max_batch-view launch sets caps the
    # server's batches below max_batch
    K = synth.default_intrinsics(160, 120)
    tr = synth.trajectory(31, 8)
    base = tg.get_schedules()
    try:
        tg.set_schedule(**{**base[8], "views_per_set": 2}, n_views=8)
        with tg.Server(max_batch=8, max_inflight=1, batch_window_us=300_000) as srv:
            bufs = {}
            for i, p in enumerate(tr):
                b = torch.zeros((120, 160, 4), dtype=torch.uint8, device=cuda)
                bufs[srv.submit(h1, p, K, 160, 120, b, client_id=i)] = (b, p)
            done = []
            while len(done) < len(tr):
                done += srv.poll(16, timeout_us=2_000_000)
        assert all(c.status == 0 for c in done)
        sets = {}
        for c in done:
            sets.setdefault((c.admit_us, c.done_us), []).append(c)
        assert max(len(v) for v in sets.values()) == 2 and len(sets) == 4
        for c in done:
            b, p = bufs[c.ticket]
            assert np.array_equal(b.cpu().numpy(), tg.render(h1, p, K, 160, 120))
    finally:
        tg.set_schedules(base)


def test_autotune_picks_a_candidate_and_keeps_frames(h1, cuda):
    levels = [(320, 240), (320, 240)]
    tr = synth.trajectory(19, 10)
    intrs = [synth.default_intrinsics(w, h) for w, h in levels]
    outs = [torch.empty((h, w, 4), dtype=torch.uint8, device=cuda) for w, h in levels]
    base = tg.get_schedules()
    try:
        marker = {"n_slices": 13, "first_slice_inv": 7, "blend_ctas_per_sm": 2, "blend_batch": 16, "views_per_set": 0}
        tg.set_schedule(**marker)
        ref = _batch(h1, tr[:2], levels, cuda)
        best, ms = tg.autotune(h1, [tr[:2], tr[4:6]], intrs, [w for w, _ in levels], [h for _, h in levels], outs,
                               iters=1)
        assert best["n_slices"] in (1, 2, 3, 4, 5, 6, 7, 8, 12)
        assert best["first_slice_inv"] in (8, 16, 32, 64, 128, 256)
        assert best["blend_ctas_per_sm"] in (0, 4) and 0 < ms < 1e4
        assert best["blend_batch"] in (16, 32) and best["views_per_set"] in (1, 2)
        # the class of two views takes the winner; a one-view winning launch set size
        # gives the one-view class the winner too; the other classes keep theirs
        assert tg.get_schedule(2) == best
        one = tg.get_schedule(1)
        if best["views_per_set"] == 1:
            assert one == {**best, "views_per_set": 0}
        else:
            assert one == marker
        assert all(tg.get_schedule(n) == marker for n in (3, 4, 8, 64))
        got = _batch(h1, tr[:2], levels, cuda)
        for a, b in zip(ref, got):
            assert np.array_equal(a, b)
    finally:
        tg.set_schedules(base)


def test_depth_sort_skips_constant_high_digit(h1, cuda):
    # a single slice: a full depth sort (no partial sort for a last slice)
    base = tg.get_schedules()
    try:
        tg.set_schedule(1, 1, 0, n_views=1)
        tg.set_schedule(1, 1, 0, n_views=2)
        # the camera at distance 3 sees depths in about [2, 4]: the kept keys span
        # far fewer than 2^24 steps, so the fourth pass is skipped
        w, h = 160, 120
        out = torch.empty((h, w, 4), dtype=torch.uint8, device=cuda)
        st = tg.render_batch(h1, [synth.BASE_POSE], [synth.default_intrinsics(w, h)], [w], [h], [out],
                             sort_mode=tg.SORT_SLICED)
        assert st["depth_sort_passes"] == 3
        assert st["depth_sort_near"] == 100_000   # every entry
        # at the edge of the scene (near plane 0.2 to depths of about 2, 2^24.8 key
        # steps in FP32 for this scene) the fourth pass runs
        inside = synth.Pose(0.0, 0.0, (0.0, 0.0, -1.0))
        st = tg.render_batch(h1, [inside], [synth.default_intrinsics(w, h)], [w], [h], [out],
                             sort_mode=tg.SORT_SLICED)
        assert st["depth_sort_passes"] == 4
        # at full size the slices' scans reuse the sort's scratch: the count is read before them
        s3 = synth.config_scene(3, n=1_000_000)
        W, H = 1920, 1080
        big = torch.empty((H, W, 4), dtype=torch.uint8, device=cuda)
        with tg.scene_from(s3, storage=tg.STORAGE_FP16) as h3:
            st = tg.render_batch(h3, [synth.config_trajectory(3)[0]] * 2, [synth.default_intrinsics(W, H)] * 2,
                                 [W] * 2, [H] * 2, [big, big], sort_mode=tg.SORT_SLICED)
        assert st["depth_sort_passes"] in (3, 4)
    finally:
        tg.set_schedules(base)


def test_partial_depth_sort_gives_the_full_sort_frames(h1, cuda):
    """Fixed-capacity launch sets of three or more slices sort by depth only
    the entries below a threshold that covers the slices before the last (a
    histogram of the depth keys places it); the last slice's pairs are
    sorted by (tile, depth key) instead.  Frames equal those of one slice (a
    full depth sort) bit for bit, whether the threshold cuts the kept entries
    (a pose that keeps most of the scene), keeps all of them (a pose that
    culls most of it, so that the slices before the last reach past the kept
    entries) or has none to keep (a camera facing away: background only)."""
    levels = [(320, 240), (160, 120)]
    poses = {"most kept": [synth.BASE_POSE, synth.trajectory(23, 5)[4]],
             "most culled": [synth.Pose(0.9, 0.0, (0.0, 0.0, -1.5)), synth.Pose(-0.9, 0.3, (0.2, 0.0, -1.5))],
             "none kept": [synth.Pose(math.pi, 0.0, (0.0, 0.0, -3.0))] * 2}
    intrs = [synth.default_intrinsics(w, hh) for w, hh in levels]
    E = 2 * 100_000
    base = tg.get_schedules()
    seen = set()
    try:
        for name, ps in poses.items():
            tg.set_schedule(1, 1, 0, n_views=2)
            ref = _batch(h1, ps, levels, cuda)
            for sch in [(3, 8, 0), (7, 128, 0), (16, 4096, 4, 16)]:
                tg.set_schedule(*sch, n_views=2)
                for _ in range(3):   # direct, exact + capture, replay
                    got = _batch(h1, ps, levels, cuda)
                    for a, b in zip(ref, got):
                        assert np.array_equal(a, b), (name, sch)
                outs = [torch.empty((hh, w, 4), dtype=torch.uint8, device=cuda) for w, hh in levels]
                for _ in range(3):   # the counting kernels' launch set, replayed on the third call
                    st = tg.render_batch(h1, ps, intrs, [w for w, _ in levels], [hh for _, hh in levels], outs,
                                         sort_mode=tg.SORT_SLICED)
                for a, b in zip(ref, outs):
                    assert np.array_equal(a, b.cpu().numpy()), (name, sch)
                S, F = sch[0], sch[1]
                first = math.ceil(F ** ((S - 2 - (S - 1)) / (S - 1)) * E)   # end of the slice before the last
                kept, near = st["n_visible"], st["depth_sort_near"]
                assert near <= kept < E
                assert near == kept or near >= first, (name, sch, near, kept, first)
                seen.add("none kept" if kept == 0 else "all kept near" if near == kept else "cut")
        assert seen == {"none kept", "all kept near", "cut"}
    finally:
        tg.set_schedules(base)