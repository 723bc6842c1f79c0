"""Pins of the JPEG oracle (CPU).

The fixed-point DCT is held to the T.81 FDCT definition; the quantizer tables
to their definition; and the bitstream is decoded by the independent decoder
in tests/jpeg_decode.py: constant images come back exactly, smooth images
within the quantization error, and the restart interval does not change any
pixel."""
import numpy as np
import pytest

from oracle import jpeg
from tests import jpeg_decode


def _ycc(rgb):
    r, g, b = [rgb[..., i].astype(np.float64) for i in range(3)]
    y = 0.299 * r + 0.587 * g + 0.114 * b
    return y, (b - y) / 1.772 + 128, (r - y) / 1.402 + 128


def test_fixed_point_dct_matches_definition():
    rng = np.random.default_rng(0)
    worst = 0.0
    for _ in range(200):
        s = rng.integers(-128, 128, (8, 8))
        got = jpeg.fdct_fixed(s) / 65536.0
        want = jpeg.fdct_exact(s)
        worst = max(worst, float(np.abs(got - want).max()))
    # weights rounded to 2^-13 (<= 8 x 128 x 2^-14 per pass) and one 2^-10 shift: well under 0.5
    assert worst < 0.25


def test_dct_of_constant_and_cosine_blocks():
    s = np.full((8, 8), 37)
    F = jpeg.fdct_exact(s)
    assert abs(F[0, 0] - 8 * 37) < 1e-9 and np.abs(F.ravel()[1:]).max() < 1e-9
    # a single basis pattern puts its energy in one coefficient; rounding its
    # samples to integers (each moved by at most 0.5) leaks less than 3 elsewhere
    x = np.arange(8)
    pat = np.round(100 * np.cos((2 * x + 1) * 3 * np.pi / 16))[None, :].repeat(8, 0)
    F = jpeg.fdct_exact(pat)
    assert abs(F[0, 3]) > 500 and np.abs(np.delete(F.ravel(), 3)).max() < 3.0


def test_quant_tables_follow_the_quality_scaling():
    base_l, base_c = jpeg.quant_table(50, False), jpeg.quant_table(50, True)
    assert base_l[0, 0] == 16 and base_l[7, 7] == 99 and base_c[0, 0] == 17 and base_c[7, 7] == 99
    assert (jpeg.quant_table(100, False) == 1).all()
    assert (jpeg.quant_table(1, True) == 255).all()
    for q in (10, 35, 65, 90):   # Table 1's qualities
        s = 5000 // q if q < 50 else 200 - 2 * q
        assert np.array_equal(jpeg.quant_table(q, False), np.clip((base_l * s + 50) // 100, 1, 255))
    qs = [jpeg.quant_table(q, False).sum() for q in range(1, 101)]
    assert all(a >= b for a, b in zip(qs, qs[1:]))


@pytest.mark.parametrize("rgb", [(0, 0, 0), (255, 255, 255), (200, 100, 50), (13, 250, 77)])
def test_constant_image_decodes_to_its_colour(rgb):
    img = np.zeros((40, 56, 4), np.uint8)
    img[..., :3] = rgb
    out = jpeg_decode.decode(jpeg.encode(img, 100))
    assert out.shape == (40, 56, 3)
    # quality 100 keeps the DC exactly; only the 8-bit YCbCr rounding remains
    assert np.abs(out - np.array(rgb)).max() <= 2.0


def _smooth(h, w, seed=1):
    y, x = np.mgrid[0:h, 0:w]
    img = np.zeros((h, w, 4), np.uint8)
    img[..., 0] = 128 + 100 * np.sin(x / 17.0 + seed)
    img[..., 1] = 128 + 90 * np.cos(y / 13.0)
    img[..., 2] = (x * 3 + y * 2) % 256 // 2 + 64
    return img


@pytest.mark.parametrize("w,h,q,floor_db", [(64, 48, 95, 35.0), (75, 37, 90, 32.0), (33, 17, 65, 27.0)])
def test_smooth_image_round_trip(w, h, q, floor_db):
    img = _smooth(h, w)
    out = jpeg_decode.decode(jpeg.encode(img, q))
    assert out.shape == (h, w, 3)
    # 4:2:0 loses chroma detail: compare luma and the 2x2-mean chroma
    y0, cb0, cr0 = _ycc(img[..., :3])
    y1, cb1, cr1 = _ycc(np.clip(np.round(out), 0, 255))
    mse = np.mean((y0 - y1) ** 2)
    assert 10 * np.log10(255 ** 2 / max(mse, 1e-12)) >= floor_db


def test_restart_interval_changes_no_pixel():
    img = _smooth(48, 80, seed=3)
    ref = jpeg_decode.decode(jpeg.encode(img, 80, restart=0))
    for r in (1, 2, 3, 7, 100):
        data = jpeg.encode(img, 80, restart=r)
        assert jpeg_decode.parse(data)["restart"] == r
        assert np.array_equal(jpeg_decode.decode(data), ref)


def test_markers_and_stuffing():
    rng = np.random.default_rng(5)
    img = rng.integers(0, 256, (32, 48, 4), dtype=np.uint8)   # noise: long codes, 0xFF bytes
    data = jpeg.encode(img, 90, restart=2)
    info = jpeg_decode.parse(data)
    assert (info["width"], info["height"]) == (48, 32)
    assert [c[:3] for c in info["comps"]] == [(1, 2, 2), (2, 1, 1), (3, 1, 1)]
    assert b"\xff\x00" in data[info["scan_start"]:]
    n_rst = sum(data.count(bytes([0xFF, 0xD0 + k]), info["scan_start"]) for k in range(8))
    assert n_rst == (3 * 2) // 2 - 1   # 6 MCUs in intervals of 2
    out = jpeg_decode.decode(data)
    assert out.shape == (32, 48, 3)
