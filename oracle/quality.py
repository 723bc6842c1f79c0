"""Reference image-quality metrics and resampler (test infrastructure).

Only the tests and bench.py's CPU legs use this module.

* ``ssim``: the structural similarity index of Wang, Bovik, Sheikh and
  Simoncelli (IEEE TIP 13(4), 2004), which Sec. 6 reports: for each colour
  channel, local means, variances and covariance under an 11 x 11 Gaussian
  window (sigma 1.5, weights normalised to 1), combined as
  ((2 mu_x mu_y + C1)(2 sigma_xy + C2)) / ((mu_x^2 + mu_y^2 + C1)(sigma_x^2 +
  sigma_y^2 + C2)) with C1 = (0.01 L)^2, C2 = (0.03 L)^2, L = 255, at every
  window position inside the image; the index is the mean over positions and
  the R, G, B channels.  FP64, separable window sums.
* ``psnr``: 10 log10(L^2 / MSE) over all pixels and the three channels.
* ``resample``: bilinear resampling with pixel centres aligned, in the 16.16
  fixed-point / 8-bit-weight integer form that the library documents.

Parity pins (tests/test_oracle_quality.py): a direct, non-separable window
sum on small images; SSIM(x, x) = 1; the closed forms for constant images,
for a luminance shift y = x + c and for the negative y = 255 - x; symmetry;
PSNR of a known error; the resampler's identity, constant and hand-worked
cases.
"""
from __future__ import annotations

import math

import numpy as np

K1, K2, L = 0.01, 0.03, 255.0
C1, C2 = (K1 * L) ** 2, (K2 * L) ** 2
WIN, SIGMA = 11, 1.5


def gaussian_1d() -> np.ndarray:
    g = np.array([math.exp(-((t - WIN // 2) ** 2) / (2 * SIGMA ** 2)) for t in range(WIN)])
    return g / g.sum()


def _filter_valid(img: np.ndarray, g: np.ndarray) -> np.ndarray:
    """sum_{s,t} g[s] g[t] img[y+s, x+t] over positions where the window fits."""
    from numpy.lib.stride_tricks import sliding_window_view
    h = sliding_window_view(img, WIN, axis=1) @ g          # [H, W-10]: rows filtered
    return sliding_window_view(h, WIN, axis=0) @ g         # [H-10, W-10]: then columns


def ssim_map(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """[3, H-10, W-10] per-channel SSIM of RGBA8 (or RGB) frames."""
    g = gaussian_1d()
    out = []
    for c in range(3):
        x = a[..., c].astype(np.float64)
        y = b[..., c].astype(np.float64)
        mx, my = _filter_valid(x, g), _filter_valid(y, g)
        sxx = _filter_valid(x * x, g) - mx * mx
        syy = _filter_valid(y * y, g) - my * my
        sxy = _filter_valid(x * y, g) - mx * my
        out.append(((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2)))
    return np.stack(out)


def ssim(a: np.ndarray, b: np.ndarray) -> float:
    return float(ssim_map(a, b).mean())


def psnr(a: np.ndarray, b: np.ndarray) -> float:
    d = a[..., :3].astype(np.float64) - b[..., :3].astype(np.float64)
    mse = float(np.mean(d * d))
    return math.inf if mse == 0 else 10 * math.log10(L * L / mse)


def _coords(n_out: int, n_in: int):
    d = np.arange(n_out, dtype=np.int64)
    c = (2 * d + 1) * n_in * 65536 // (2 * n_out) - 32768
    c = np.maximum(c, 0)
    i0 = c >> 16
    f = (c >> 8) & 255
    edge = i0 >= n_in - 1
    i0 = np.where(edge, n_in - 1, i0)
    f = np.where(edge, 0, f)
    i1 = np.minimum(i0 + 1, n_in - 1)
    return i0, i1, f


def resample(src: np.ndarray, width: int, height: int) -> np.ndarray:
    """Bilinear RGBA8 resample of src [h, w, 4] to [height, width, 4]."""
    h, w = src.shape[:2]
    x0, x1, fx = _coords(width, w)
    y0, y1, fy = _coords(height, h)
    s = src.astype(np.int64)
    fx = fx[None, :, None]
    fy = fy[:, None, None]
    top = s[y0][:, x0] * (256 - fx) + s[y0][:, x1] * fx
    bot = s[y1][:, x0] * (256 - fx) + s[y1][:, x1] * fx
    return np.ascontiguousarray(((top * (256 - fy) + bot * fy + 32768) >> 16).astype(np.uint8))
