"""Pins of the quality oracle (oracle/quality.py) on the CPU."""
import math

import numpy as np
import pytest

from oracle import quality as q


def _img(h, w, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 256, (h, w, 4), dtype=np.uint8)


def _smooth(h, w, seed):
    y, x = np.mgrid[0:h, 0:w]
    img = np.zeros((h, w, 4), np.uint8)
    img[..., 0] = 128 + 90 * np.sin(x / 7.0 + seed)
    img[..., 1] = 128 + 80 * np.cos(y / 5.0 - seed)
    img[..., 2] = (x * 5 + y * 3 + 17 * seed) % 200 + 20
    img[..., 3] = 255
    return img


def test_window_is_the_normalised_gaussian():
    g = q.gaussian_1d()
    assert abs(g.sum() - 1) < 1e-15 and np.allclose(g, g[::-1])
    assert abs(g[5] / g[6] - math.exp(1 / (2 * 1.5 ** 2))) < 1e-12


def test_separable_sums_match_a_direct_window_sum():
    """Brute force: the 121-tap 2-D window summed directly, per position."""
    a, b = _img(14, 17, 1), _img(14, 17, 2)
    g = q.gaussian_1d()
    w2 = np.outer(g, g)
    got = q.ssim_map(a, b)
    for c in range(3):
        x, y = a[..., c].astype(float), b[..., c].astype(float)
        for i in range(14 - 10):
            for j in range(17 - 10):
                X, Y = x[i:i + 11, j:j + 11], y[i:i + 11, j:j + 11]
                mx, my = (w2 * X).sum(), (w2 * Y).sum()
                vx = (w2 * (X - mx) ** 2).sum()
                vy = (w2 * (Y - my) ** 2).sum()
                cxy = (w2 * (X - mx) * (Y - my)).sum()
                want = ((2 * mx * my + q.C1) * (2 * cxy + q.C2)) / ((mx ** 2 + my ** 2 + q.C1) * (vx + vy + q.C2))
                assert abs(got[c, i, j] - want) < 1e-12


def test_identical_frames():
    a = _img(40, 33, 3)
    assert abs(q.ssim(a, a) - 1.0) < 1e-12
    assert q.psnr(a, a) == math.inf


@pytest.mark.parametrize("u,v", [(0, 255), (10, 200), (128, 129), (77, 77)])
def test_constant_frames_closed_form(u, v):
    a = np.full((20, 23, 4), u, np.uint8)
    b = np.full((20, 23, 4), v, np.uint8)
    want = (2 * u * v + q.C1) / (u * u + v * v + q.C1)
    assert np.allclose(q.ssim_map(a, b), want, atol=1e-12)


def test_luminance_shift_closed_form():
    """y = x + c: sigma_y = sigma_x = sigma_xy, so only the luminance term remains."""
    a = _smooth(30, 31, 1)
    a[..., :3] = a[..., :3] // 2 + 20          # room for the shift
    c = 37
    b = a.copy()
    b[..., :3] += c
    g = q.gaussian_1d()
    got = q.ssim_map(a, b)
    for ch in range(3):
        mx = q._filter_valid(a[..., ch].astype(float), g)
        want = (2 * mx * (mx + c) + q.C1) / (mx ** 2 + (mx + c) ** 2 + q.C1)
        assert np.allclose(got[ch], want, atol=1e-10)


def test_negative_closed_form():
    """y = 255 - x: sigma_y = sigma_x and sigma_xy = -sigma_x^2."""
    a = _smooth(26, 29, 2)
    b = a.copy()
    b[..., :3] = 255 - a[..., :3]
    g = q.gaussian_1d()
    got = q.ssim_map(a, b)
    for ch in range(3):
        x = a[..., ch].astype(float)
        mx = q._filter_valid(x, g)
        vx = q._filter_valid(x * x, g) - mx ** 2
        my = 255 - mx
        want = ((2 * mx * my + q.C1) * (-2 * vx + q.C2)) / ((mx ** 2 + my ** 2 + q.C1) * (2 * vx + q.C2))
        assert np.allclose(got[ch], want, atol=1e-9)


def test_symmetry_and_range():
    a, b = _img(25, 30, 5), _smooth(25, 30, 3)
    assert abs(q.ssim(a, b) - q.ssim(b, a)) < 1e-14
    m = q.ssim_map(a, b)
    assert (m <= 1 + 1e-12).all() and (m >= -1 - 1e-12).all()


def test_psnr_of_a_known_error():
    a = np.full((8, 8, 4), 100, np.uint8)
    b = a.copy()
    b[0, 0, 0] = 110     # one sample off by 10: MSE = 100 / 192
    assert abs(q.psnr(a, b) - 10 * math.log10(255 ** 2 * 192 / 100)) < 1e-12
    b[..., 3] = 0        # alpha is ignored
    assert abs(q.psnr(a, b) - 10 * math.log10(255 ** 2 * 192 / 100)) < 1e-12


def test_resample_identity_and_constant():
    a = _img(13, 21, 7)
    assert np.array_equal(q.resample(a, 21, 13), a)
    c = np.full((5, 9, 4), 173, np.uint8)
    assert (q.resample(c, 31, 17) == 173).all() and (q.resample(c, 3, 2) == 173).all()


def test_resample_hand_worked_2x():
    """2 x 2 -> 4 x 4: centres at s = -0.25 (clamped to 0), 0.25, 0.75, 1.25 (edge)."""
    src = np.zeros((2, 2, 4), np.uint8)
    src[..., 0] = [[0, 200], [100, 40]]
    out = q.resample(src, 4, 4)[..., 0].astype(int)
    # weights along each axis: 0, 64, 192, edge -> (0|64|192)/256 of the next sample
    def lerp(p, r, f):
        return int(p) * (256 - f) + int(r) * f
    fs = [0, 64, 192, 0]
    idx = [0, 0, 0, 1]
    for i in range(4):
        for j in range(4):
            y0, x0 = idx[i], idx[j]
            y1, x1 = min(y0 + 1, 1), min(x0 + 1, 1)
            t = lerp(src[y0, x0, 0], src[y0, x1, 0], fs[j])
            b = lerp(src[y1, x0, 0], src[y1, x1, 0], fs[j])
            assert out[i, j] == (t * (256 - fs[i]) + b * fs[i] + 32768) >> 16
    assert out[0, 0] == 0 and out[0, 3] == 200 and out[3, 0] == 100 and out[3, 3] == 40
    # the 0.25 / 0.75 interior: 0.75 * 0 + 0.25 * 200 = 50 along the top row
    assert out[0, 1] == 50 and out[0, 2] == 150


def test_constants_of_the_published_index():
    """K1 = 0.01, K2 = 0.03, L = 255 and an 11 x 11, sigma 1.5 window (Wang et al. 2004)."""
    assert q.C1 == pytest.approx(6.5025, abs=1e-12) and q.C2 == pytest.approx(58.5225, abs=1e-12)
    assert q.WIN == 11 and q.SIGMA == 1.5
    # black against white: only the luminance term differs from 1
    a = np.zeros((11, 11, 4), np.uint8)
    b = np.full((11, 11, 4), 255, np.uint8)
    assert q.ssim(a, b) == pytest.approx(6.5025 / (255 ** 2 + 6.5025), rel=1e-12)
