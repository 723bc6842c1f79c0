"""Pins for the oracle's EWA projection, culling, compositing and tile lists.

Closed forms (single Gaussians), invariants (zero opacity, alpha channel,
permutations, transmittance stop), brute force on tiny scenes, and the
brute-force tile enumeration.
"""
import math

import numpy as np
import pytest

import oracle
import synth

C0 = 0.28209479177387814


def scene_of(mus, log_scales, quats, logits, dcs):
    n = len(mus)
    sh = np.zeros((n, 16, 3), np.float32)
    sh[:, 0, :] = np.asarray(dcs, np.float32)
    return synth.Scene(np.asarray(mus, np.float32), np.asarray(log_scales, np.float32),
                       np.asarray(quats, np.float32), np.asarray(logits, np.float32), sh, 0)


def _iso(mu, sigma, logit, dc):
    ls = math.log(sigma)
    return scene_of([mu], [[ls] * 3], [[1, 0, 0, 0]], [logit], [dc])


def test_isotropic_gaussian_closed_form_footprint():
    # on the optical axis at depth z: Sigma2 = ((f s / z)^2 + 0.3) I, alpha(d) =
    # min(0.99, o exp(-|d|^2 / (2 var))) inside the tile support, pixel = alpha c
    W, H = 97, 81
    K = synth.Intrinsics(120.0, 120.0, W / 2, H / 2)
    sigma, logit, dc = 0.05, 0.8, (0.3, -0.1, 0.9)
    sc = _iso((0.0, 0.0, 0.0), sigma, logit, dc)
    pr = oracle.preprocess(sc, synth.BASE_POSE, K, W, H)
    z = 3.0
    s32 = math.exp(float(np.float32(math.log(sigma))))
    var = (120.0 * s32 / z) ** 2 + 0.3
    o = 1.0 / (1.0 + math.exp(-float(np.float32(logit))))
    assert np.allclose(pr.conic[0], [1 / var, 0.0, 1 / var], rtol=1e-13)
    r = math.ceil(3 * math.sqrt(var))
    assert pr.radius[0] == r
    img = oracle.render(pr)
    col = np.maximum(0, 0.5 + C0 * np.array(dc, np.float32).astype(np.float64))
    TX, TY = pr.tiles_xy
    x0, x1 = max(0, math.floor((W / 2 - r) / 16)), min(TX, math.floor((W / 2 + r) / 16) + 1)
    y0, y1 = max(0, math.floor((H / 2 - r) / 16)), min(TY, math.floor((H / 2 + r) / 16) + 1)
    assert tuple(pr.rect[0]) == (x0, y0, x1, y1)
    for j in range(H):
        for i in range(W):
            inside = x0 <= i // 16 < x1 and y0 <= j // 16 < y1
            d2 = (i + 0.5 - W / 2) ** 2 + (j + 0.5 - H / 2) ** 2
            a = min(0.99, o * math.exp(-d2 / (2 * var)))
            if not inside or a < 1 / 255:
                a = 0.0
            assert np.allclose(img[j, i, :3], a * col, atol=1e-12, rtol=0)
            assert abs(img[j, i, 3] - a) < 1e-12


def test_off_axis_jacobian_closed_form():
    # isotropic Gaussian at camera point (x, 0, z): J = [[f/z, 0, -f x/z^2],[0, f/z, 0]]
    # so Sigma2 = s^2 J J^T + 0.3 I = diag(s^2 f^2 (1/z^2 + x^2/z^4), s^2 f^2/z^2) + 0.3
    W, H = 200, 200
    f = 150.0
    K = synth.Intrinsics(f, f, 100.0, 100.0)
    x = 0.9
    sc = _iso((x, 0.0, 0.0), 0.04, 1.0, (0, 0, 0))
    pr = oracle.preprocess(sc, synth.BASE_POSE, K, W, H)
    z = 3.0
    s = math.exp(float(np.float32(math.log(0.04))))
    x32 = float(np.float32(x))
    a = s * s * f * f * (1 / z ** 2 + x32 ** 2 / z ** 4) + 0.3
    c = s * s * f * f / z ** 2 + 0.3
    assert np.allclose(pr.conic[0], [1 / a, 0.0, 1 / c], rtol=1e-12, atol=1e-15)
    # beyond the 1.3 x half-FOV guard band the Jacobian uses the clamped point
    x_far = 3.0 * 1.3 * (W / (2 * f)) * z
    pr2 = oracle.preprocess(_iso((x_far, 0.0, 0.0), 0.04, 1.0, (0, 0, 0)), synth.BASE_POSE, K, W, H)
    tx = 1.3 * W / (2 * f) * z
    a2 = s * s * f * f * (1 / z ** 2 + tx ** 2 / z ** 4) + 0.3
    assert abs(pr2.conic[0, 0] - 1 / a2) < 1e-12 * (1 / a2)


def test_quaternion_rotation_about_view_axis():
    # q = (cos(psi/2), 0, 0, sin(psi/2)) turns the x axis towards y by psi:
    # Sigma2 = (f/z)^2 R_psi diag(s1^2, s2^2) R_psi^T + 0.3 I
    W = H = 128
    f = 100.0
    K = synth.Intrinsics(f, f, 64.0, 64.0)
    psi = 0.6
    ls = [math.log(0.08), math.log(0.02), math.log(0.05)]
    q = [math.cos(psi / 2), 0.0, 0.0, math.sin(psi / 2)]
    sc = scene_of([(0, 0, 0)], [ls], [q], [1.0], [(0, 0, 0)])
    pr = oracle.preprocess(sc, synth.BASE_POSE, K, W, H)
    s1, s2 = (math.exp(float(np.float32(v))) for v in ls[:2])
    q32 = np.array(q, np.float32).astype(np.float64)
    q32 /= np.linalg.norm(q32)
    ps = 2 * math.atan2(q32[3], q32[0])
    Rp = np.array([[math.cos(ps), -math.sin(ps)], [math.sin(ps), math.cos(ps)]])
    S2 = (f / 3.0) ** 2 * Rp @ np.diag([s1 * s1, s2 * s2]) @ Rp.T + 0.3 * np.eye(2)
    Ci = np.linalg.inv(S2)
    assert np.allclose(pr.conic[0], [Ci[0, 0], Ci[0, 1], Ci[1, 1]], rtol=1e-11, atol=1e-14)
    # the major axis direction follows the sign convention of the rotation
    assert pr.conic[0, 1] < 0   # Sigma2 off-diagonal > 0 for psi in (0, pi/2)
    lam = 0.5 * (S2[0, 0] + S2[1, 1]) + math.sqrt(max(0.1, (0.5 * (S2[0, 0] - S2[1, 1])) ** 2 + S2[0, 1] ** 2))
    assert pr.radius[0] == math.ceil(3 * math.sqrt(lam))


def test_near_plane_and_opacity_culls():
    K = synth.default_intrinsics(64, 64)
    sc = scene_of([(0, 0, -2.85), (0, 0, -2.75), (0, 0, 0), (0, 0, 0)],
                  [[-3.0] * 3] * 4, [[1, 0, 0, 0]] * 4,
                  [2.0, 2.0, math.log((1 / 255 * 0.99) / (1 - 1 / 255 * 0.99)),
                   math.log((1 / 255 * 1.01) / (1 - 1 / 255 * 1.01))], [(0, 0, 0)] * 4)
    pr = oracle.preprocess(sc, synth.BASE_POSE, K, 64, 64)
    assert pr.cull.tolist() == [1, 0, 2, 0]          # z = 0.15 culled, z = 0.25 kept
    assert pr.visible.tolist() == [0, 1, 0, 1]


def test_frustum_cull_by_empty_rect():
    K = synth.default_intrinsics(64, 64)
    sc = scene_of([(5.0, 0, 0), (0, 0, 0)], [[-5.0] * 3] * 2, [[1, 0, 0, 0]] * 2, [2.0, 2.0], [(0, 0, 0)] * 2)
    pr = oracle.preprocess(sc, synth.BASE_POSE, K, 64, 64)
    assert pr.cull.tolist() == [4, 0] and pr.tiles_touched.tolist()[0] == 0


def test_zero_opacity_gives_background_exactly():
    s = synth.config_scene(1, n=3000)
    s.opacity_logits[:] = -40.0
    bg = (0.2, 0.4, 0.6)
    pr = oracle.preprocess(s, synth.BASE_POSE, synth.default_intrinsics(64, 48), 64, 48)
    img = oracle.render(pr, background=bg)
    assert np.all(img[..., :3] == np.array(bg)) and np.all(img[..., 3] == 0.0)


def _stack(opacities, colours, W=33, H=33):
    # Gaussians on the optical axis at increasing depth; odd W, H put a pixel
    # centre exactly on the axis, where power = 0 and alpha = min(0.99, o)
    n = len(opacities)
    mus = [(0.0, 0.0, 0.1 * k) for k in range(n)]
    logits = [math.log(o / (1 - o)) if o < 1 else 40.0 for o in opacities]
    dcs = [tuple((np.array(c) - 0.5) / C0) for c in colours]
    sc = scene_of(mus, [[-3.0] * 3] * n, [[1, 0, 0, 0]] * n, logits, dcs)
    K = synth.Intrinsics(40.0, 40.0, W / 2, H / 2)
    return oracle.preprocess(sc, synth.BASE_POSE, K, W, H)


def test_alpha_channel_product_and_front_to_back_order():
    ops = [0.3, 0.5, 0.25]
    cols = [(1, 0, 0), (0, 1, 0), (0, 0, 1)]
    pr = _stack(ops, cols)
    px = oracle.render(pr, pixels=[(16, 16)])[0]
    a = np.array([pr.opacity[k] for k in range(3)])
    T = 1.0
    C = np.zeros(3)
    for k in range(3):
        C += np.array(pr.rgb[k]) * a[k] * T
        T *= 1 - a[k]
    assert np.allclose(px[:3], C, atol=1e-14)
    assert abs(px[3] - (1 - np.prod(1 - a))) < 1e-14
    # the nearest Gaussian gets the largest weight
    assert px[0] > px[1] * 0.3 / (0.5 * 0.7) * 0.999


def test_alpha_cap_and_transmittance_stop():
    # o = 1 gives alpha = 0.99; two such Gaussians leave T = 1e-4 (blended, since
    # the stop test is T < 1e-4), a third would bring T to 1e-6: not blended
    pr = _stack([1.0, 1.0, 1.0], [(1, 0, 0), (0, 1, 0), (0, 0, 1)])
    px, ev = oracle.render(pr, pixels=[(16, 16)], want_evals=True)
    expect = np.array([0.99, 0.99 * (1 - 0.99), 0.0])
    assert np.allclose(px[0, :3], expect, atol=1e-12)
    assert ev[0] == 3
    assert abs(px[0, 3] - (1 - (1 - 0.99) ** 2)) < 1e-12


def test_two_opaque_gaussians_nearer_wins():
    pr = _stack([0.999, 0.999], [(0.1, 0.8, 0.3), (0.9, 0.2, 0.6)])
    px = oracle.render(pr, pixels=[(16, 16)])[0]
    assert np.allclose(px[:3], 0.99 * np.array(pr.rgb[0]) + 0.99 * 0.01 * np.array(pr.rgb[1]), atol=1e-12)


def test_transmittance_monotone_along_list():
    s = synth.config_scene(1, n=20000)
    pr = oracle.preprocess(s, synth.BASE_POSE, synth.default_intrinsics(64, 48), 64, 48)
    order = np.argsort(pr.uvz[:, 2], kind="stable")
    prev = None
    for m in [50, 200, 1000, 5000, 20000]:
        keep = np.zeros(pr.visible.shape, bool)
        keep[order[:m]] = True                      # nearest m Gaussians only
        sub = oracle.Projected(**{**pr.__dict__, "visible": (pr.visible * keep).astype(np.int8)})
        a = oracle.render(sub)[..., 3]
        if prev is not None:
            assert np.all(a >= prev - 1e-15)       # 1 - T never decreases with more Gaussians
        prev = a


def test_permutation_invariance():
    s = synth.config_scene(1, n=4000)
    K = synth.default_intrinsics(80, 60)
    pose = synth.Pose(0.1, 0.05, (0.02, 0.0, -3.0))
    img = oracle.render(oracle.preprocess(s, pose, K, 80, 60))
    perm = np.random.default_rng(0).permutation(s.n)
    img2 = oracle.render(oracle.preprocess(s.subset(perm), pose, K, 80, 60))
    assert np.array_equal(img, img2)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tile_grouping_equals_brute_force(seed):
    s = synth.make_scene(64, 1000 + seed, n_blobs=4, iso_sigma=0.2)
    s.log_scales += 1.0                             # larger footprints on a 32x32 frame
    pose = synth.Pose(0.05 * seed, -0.03, (0.0, 0.0, -2.5))
    pr = oracle.preprocess(s, pose, synth.default_intrinsics(32, 32), 32, 32)
    a = oracle.render(pr, background=(0.1, 0.2, 0.3))
    b = oracle.render_brute(pr, background=(0.1, 0.2, 0.3))
    assert np.array_equal(a, b)
    pix = [(3, 4), (31, 0), (16, 16), (0, 31)]
    c = oracle.render(pr, background=(0.1, 0.2, 0.3), pixels=pix)
    assert np.array_equal(c, np.array([b[y, x] for x, y in pix]))


def support_rule_scene():
    """One isotropic, nearly opaque Gaussian whose alpha >= 1/255 region reaches
    past its 3-sigma tile rectangle: on a 64x32 frame (f = 120, centre (32, 16))
    it projects to u = 32.9 with 3 sqrt(lambda) = 14.9, so r = 15 and
    x_hi = floor((u + r) / 16) + 1 = 3, while the centre of pixel 48 (tile 3)
    lies 15.6 px from u, where alpha = 0.99 exp(-15.6^2 / (2 (14.9 / 3)^2))
    ~ 7e-3 > 1/255."""
    W, H = 64, 32
    K = synth.Intrinsics(120.0, 120.0, W / 2, H / 2)
    s_px = math.sqrt((14.9 / 3) ** 2 - 0.3)          # pixel sigma before the 0.3 dilation
    scale = s_px * 3.0 / 120.0                       # at depth 3
    sc = scene_of([(0.9 * 3.0 / 120.0, 0.0, 0.0)], [[math.log(scale)] * 3], [[1, 0, 0, 0]], [5.0],
                  [(1.0, 1.0, 1.0)])
    return sc, K, W, H


def test_support_rule_changes_a_named_pixel():
    # the tiled method composites a Gaussian only in the tiles of its rectangle;
    # the plain per-pixel definition includes that rule (else parity would fail
    # by construction), and this scene shows the rule is not vacuous
    sc, K, W, H = support_rule_scene()
    pr = oracle.preprocess(sc, synth.BASE_POSE, K, W, H)
    assert pr.radius[0] == 15 and tuple(pr.rect[0]) == (1, 0, 3, 2)
    u, v = pr.uvz[0, 0], pr.uvz[0, 1]
    assert abs(u - 32.9) < 1e-6 and abs(v - 16.0) < 1e-9
    with_rule = oracle.render_brute(pr)
    without = oracle.render_brute(pr, support_rule=False)
    assert np.array_equal(oracle.render(pr), with_rule)
    # pixel (48, 16): outside the rectangle, so exactly the (black) background with the rule ...
    assert np.all(with_rule[16, 48] == 0.0)
    # ... and alpha = min(0.99, o exp(-q/2)) > 1/255 without it, q from the conic at the pixel centre
    A, B, C = pr.conic[0]
    dx, dy = 48.5 - u, 16.5 - v
    o = 1.0 / (1.0 + math.exp(-5.0))
    alpha = min(0.99, o * math.exp(-0.5 * (A * dx * dx + 2 * B * dx * dy + C * dy * dy)))
    assert 1 / 255 < alpha < 0.01
    assert abs(without[16, 48, 3] - alpha) < 1e-12
    col = 0.5 + C0 * float(np.float32(1.0))
    assert np.allclose(without[16, 48, :3], alpha * col, atol=1e-12)
    # inside the rectangle (pixel 47) the two agree; the rule changes only tile-3 pixels
    assert np.array_equal(with_rule[:, :48], without[:, :48])
    assert np.any(without[:, 48:] != with_rule[:, 48:])


def test_tile_lists_equal_brute_enumeration():
    s = synth.config_scene(1, n=3000)
    pr = oracle.preprocess(s, synth.Pose(0.1, 0.0, (0, 0, -3.0)), synth.default_intrinsics(120, 90), 120, 90)
    ranges, values = oracle.tile_lists(pr)
    TX, TY = pr.tiles_xy
    assert ranges[-1, 1] == oracle.pair_count(pr) == pr.tiles_touched.sum()
    assert np.array_equal(ranges[1:, 0], ranges[:-1, 1]) and ranges[0, 0] == 0
    for t in range(TX * TY):
        tx, ty = t % TX, t // TX
        members = [i for i in range(s.n) if pr.visible[i] and pr.rect[i, 0] <= tx < pr.rect[i, 2]
                   and pr.rect[i, 1] <= ty < pr.rect[i, 3]]
        members.sort(key=lambda i: (pr.uvz[i, 2], i))
        assert values[ranges[t, 0]:ranges[t, 1]].tolist() == members
        if t % 7 == 0:
            assert oracle.tile_list(pr, tx, ty).tolist() == members


def test_guard_band_candidates_cover_decision():
    s = synth.config_scene(1, n=20000)
    pr = oracle.preprocess(s, synth.BASE_POSE, synth.default_intrinsics(320, 240), 320, 240)
    v = pr.visible > 0
    c = pr.cand
    assert np.all((c[v, 2] <= pr.radius[v]) & (pr.radius[v] <= c[v, 3]))
    for k, col in enumerate([0, 1, 2, 3]):
        lo, hi = c[v, 4 + 2 * k], c[v, 5 + 2 * k]
        x = pr.rect[v, [0, 1, 2, 3][k]]
        assert np.all((lo <= x) & (x <= hi))
    # non-ambiguous Gaussians have a single candidate everywhere
    na = v & (pr.amb == 0)
    assert np.all(c[na, 2] == c[na, 3]) and np.all(c[na, 4] == c[na, 5])
    assert 0 < pr.amb.sum() < 0.01 * s.n


def test_fp16_storage_model_changes_little():
    s = synth.config_scene(1, n=20000)
    K = synth.default_intrinsics(160, 120)
    a = oracle.render(oracle.preprocess(s, synth.BASE_POSE, K, 160, 120))
    b = oracle.render(oracle.preprocess(s, synth.BASE_POSE, K, 160, 120, storage_half=True))
    assert 0 < np.abs(a - b).max() < 0.2
    assert oracle.psnr(a[..., :3], b[..., :3]) > 40
