"""Pins for the oracle's camera model, intrinsics scaling and SH basis.

Each check compares against something other than the oracle's own formula:
rigid-motion invariants, closed-form projections, quadrature, the addition
theorem, and scipy's complex spherical harmonics.
"""
import math

import numpy as np
import pytest
import scipy.special as ss

import oracle
import synth


def _one_gaussian(mu, log_scale=(-4.0, -4.0, -4.0), quat=(1, 0, 0, 0), logit=2.0, dc=(0.1, 0.2, 0.3)):
    sh = np.zeros((1, 16, 3), np.float32)
    sh[0, 0] = dc
    return synth.Scene(np.array([mu], np.float32), np.array([log_scale], np.float32),
                       np.array([quat], np.float32), np.array([logit], np.float32), sh, 0)


@pytest.mark.parametrize("az,el", [(0.0, 0.0), (0.7, -0.3), (-2.1, 1.2), (3.0, 0.9)])
def test_rotation_is_proper_and_forward_axis(az, el):
    R = oracle.camera_rotation(az, el)
    assert np.allclose(R @ R.T, np.eye(3), atol=1e-14)
    assert abs(np.linalg.det(R) - 1.0) < 1e-14
    fwd = np.array([math.sin(az) * math.cos(el), -math.sin(el), math.cos(az) * math.cos(el)])
    assert np.allclose(R[:, 2], fwd, atol=1e-14)
    # azimuth turns about the world y axis only: the right axis stays horizontal
    assert abs(R[1, 0]) < 1e-14


def test_world_to_camera_is_rigid_and_maps_centre_to_origin():
    rng = np.random.default_rng(0)
    t = rng.normal(size=3)
    T = oracle.world_to_camera(0.4, -0.2, t)
    assert np.allclose(T[3], [0, 0, 0, 1])
    assert np.allclose(T @ np.append(t, 1.0), [0, 0, 0, 1], atol=1e-14)
    p, q = rng.normal(size=3), rng.normal(size=3)
    pc, qc = T @ np.append(p, 1), T @ np.append(q, 1)
    assert abs(np.linalg.norm(pc[:3] - qc[:3]) - np.linalg.norm(p - q)) < 1e-13


@pytest.mark.parametrize("az,el,d", [(0.0, 0.0, 3.0), (0.5, 0.2, 2.0), (-1.0, -0.6, 4.5)])
def test_point_on_forward_axis_projects_to_principal_point(az, el, d):
    t = np.array([0.1, -0.2, -3.0])
    fwd = oracle.camera_rotation(az, el)[:, 2]
    pose = synth.Pose(az, el, tuple(t))
    K = synth.default_intrinsics(321, 241)
    pr = oracle.preprocess(_one_gaussian(t + d * fwd), pose, K, 321, 241)
    u, v, z = pr.uvz[0]
    # the mean is stored as float32 (rounding ~3e-7), hence the tolerances
    assert abs(u - K.cx) < 1e-4 and abs(v - K.cy) < 1e-4 and abs(z - d) < 1e-6


def test_pinhole_projection_closed_form():
    # camera at the base pose: p_c = mu - t, so u = fx x/z + cx, v = fy y/z + cy
    K = synth.Intrinsics(300.0, 280.0, 150.0, 110.0)
    mu = (0.3, -0.2, 0.5)
    pr = oracle.preprocess(_one_gaussian(mu), synth.BASE_POSE, K, 300, 220)
    z = 3.5
    assert np.allclose(pr.uvz[0], [300 * 0.3 / z + 150, 280 * -0.2 / z + 110, z], atol=1e-12)


def test_intrinsics_scaling_keeps_view():
    # Sec. 5.3: on a resolution change fx, fy, cx, cy scale with the frame so the
    # FoV stays fixed; projected centres then scale by the same factor.
    s = synth.config_scene(1, n=2000)
    pose = synth.Pose(0.2, -0.1, (0.05, 0.02, -2.9))
    K = synth.default_intrinsics(1920, 1080)
    base = oracle.preprocess(s, pose, K, 1920, 1080)
    for f in [0.25, 0.4, 0.5, 2 / 3, 0.8]:
        w, h = round(1920 * f), round(1080 * f)
        pr = oracle.preprocess(s, pose, synth.scale_intrinsics(K, w / 1920, h / 1080), w, h)
        m = (base.visible > 0) & (pr.visible > 0)
        assert m.sum() > 1000
        assert np.allclose(pr.uvz[m, 0], base.uvz[m, 0] * w / 1920, rtol=0, atol=1e-9)
        assert np.allclose(pr.uvz[m, 1], base.uvz[m, 1] * h / 1080, rtol=0, atol=1e-9)


# ------------------------------------------------------------------- SH


def _sphere_quadrature(n_theta=48, n_phi=96):
    x, w = np.polynomial.legendre.leggauss(n_theta)          # cos(theta) nodes
    ph = (np.arange(n_phi) + 0.5) * 2 * math.pi / n_phi
    dirs, wts = [], []
    for xi, wi in zip(x, w):
        st = math.sqrt(1 - xi * xi)
        for p in ph:
            dirs.append((st * math.cos(p), st * math.sin(p), xi))
            wts.append(wi * 2 * math.pi / n_phi)
    return np.array(dirs), np.array(wts)


def test_sh_orthonormal_by_quadrature():
    dirs, wts = _sphere_quadrature()
    Y = np.array([oracle.sh_basis(d) for d in dirs])       # [Q,16]
    G = (Y * wts[:, None]).T @ Y
    assert np.allclose(G, np.eye(16), atol=1e-10)


def test_sh_addition_theorem_and_parity():
    rng = np.random.default_rng(1)
    for _ in range(50):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        Y, Ym = oracle.sh_basis(d), oracle.sh_basis(-d)
        for l in range(4):
            band = Y[l * l:(l + 1) ** 2]
            assert abs(np.sum(band ** 2) - (2 * l + 1) / (4 * math.pi)) < 1e-12
            assert np.allclose(Ym[l * l:(l + 1) ** 2], (-1) ** l * band, atol=1e-14)


def test_sh_matches_scipy_complex_harmonics():
    # real form from the complex Y_l^m (Condon-Shortley phase, as in scipy):
    #   m > 0: sqrt2 Re Y_l^m;  m < 0: sqrt2 Im Y_l^|m|;  m = 0: Y_l^0
    rng = np.random.default_rng(2)
    for _ in range(40):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        th, ph = math.acos(d[2]), math.atan2(d[1], d[0])
        Y = oracle.sh_basis(d)
        for l in range(4):
            for m in range(-l, l + 1):
                c = complex(ss.sph_harm_y(l, abs(m), th, ph))
                ref = c.real if m == 0 else math.sqrt(2) * (c.real if m > 0 else c.imag)
                assert abs(Y[l * l + l + m] - ref) < 1e-13


def test_sh_degree1_linear_form_and_pole_values():
    c1 = math.sqrt(3 / (4 * math.pi))
    rng = np.random.default_rng(3)
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    Y = oracle.sh_basis(d)
    assert np.allclose(Y[1:4], [-c1 * d[1], c1 * d[2], -c1 * d[0]], atol=1e-15)
    Yp = oracle.sh_basis([0.0, 0.0, 1.0])
    for l in range(4):
        for m in range(-l, l + 1):
            expect = math.sqrt((2 * l + 1) / (4 * math.pi)) if m == 0 else 0.0
            assert abs(Yp[l * l + l + m] - expect) < 1e-15
    assert np.all(oracle.sh_basis(d, degree=1)[4:] == 0.0)


def test_sh_degree0_colour_rule():
    # degree 0 (the paper's default, Sec. 5.1): colour = 0.5 + C0 f_dc, clamped at 0
    C0 = 0.28209479177387814
    assert abs(oracle.sh_basis([1.0, 0.0, 0.0])[0] - C0) < 1e-16
    for dc in [(0.1, -0.4, 2.0), (-3.0, 0.0, 0.7)]:
        pr = oracle.preprocess(_one_gaussian((0.0, 0.0, 0.0), dc=dc), synth.BASE_POSE,
                               synth.default_intrinsics(64, 64), 64, 64)
        assert np.allclose(pr.rgb[0], np.maximum(0.0, 0.5 + C0 * np.array(dc, np.float32)), atol=1e-15)


def test_sh_rotation_consistency_degree1():
    # rotating the view direction and the degree-1 coefficients together leaves
    # the colour unchanged (degree-1 coefficients transform like a vector)
    rng = np.random.default_rng(4)
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    a = rng.normal(size=3)                  # value = a . (-y, z, -x) * c1
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    to_vec = lambda c: np.array([-c[2], -c[0], c[1]])     # (c_{1,-1}, c_{10}, c_{11}) -> vector
    from_vec = lambda v: np.array([-v[1], v[2], -v[0]])
    val = oracle.sh_basis(d)[1:4] @ a
    a_rot = from_vec(Q @ to_vec(a))
    val_rot = oracle.sh_basis(Q @ d)[1:4] @ a_rot
    assert abs(val - val_rot) < 1e-14


# -------------------------------------------------------------- fp16 model


def test_round_half_matches_numpy_binary16():
    rng = np.random.default_rng(5)
    xs = np.concatenate([rng.normal(size=2000) * 10.0 ** rng.integers(-9, 4, size=2000),
                         [0.0, 1.0, 65504.0, 6.1e-5, 5.96e-8, 1 + 2 ** -11, 1 + 3 * 2 ** -11]])
    for x in xs:
        assert oracle.round_half(x) == float(np.float64(x).astype(np.float16))


def test_rgba8_rounding():
    v = np.array([[0.0, 1.0, -0.5, 2.0], [0.5 / 255, 1.5 / 255, 0.49 / 255, 254.5 / 255]])
    assert oracle.to_rgba8(v).tolist() == [[0, 255, 0, 255], [1, 2, 0, 255]]
