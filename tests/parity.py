"""Parity helpers shared by the GPU tests: compare the CUDA path with the oracle.

Integer work (culling, radius, tile rectangle, per-tile lists, ranges) must be
bit-exact on every Gaussian whose FP64 decisions lie outside the oracle's
guard bands; an ambiguous Gaussian must take one of the outcomes the oracle
lists for it.  Within a tile, two Gaussians whose FP64 depths differ by less
than DEPTH_TIE_REL (relative) may appear in either order.

Colour gate (float RGBA before 8-bit encoding): max |d| <= 2e-3 on at least
99.9 % of pixels, mean |d| <= 1e-4, PSNR >= 50 dB.
"""
from __future__ import annotations

import numpy as np

import oracle

DEPTH_TIE_REL = 2.0 ** -20
COLOUR_MAX_ABS = 2e-3
COLOUR_FRACTION = 0.999
COLOUR_MEAN_ABS = 1e-4
PSNR_MIN_DB = 50.0


def check_per_gaussian(dbg: dict, pr: oracle.Projected) -> dict:
    """Culled set, radius and rect: exact off the guard bands, a candidate on them."""
    amb = pr.amb > 0
    vis_g = dbg["visible"].astype(np.int32)
    vis_o = pr.visible.astype(np.int32)
    na = ~amb
    bad_vis = np.nonzero(na & (vis_g != vis_o))[0]
    assert bad_vis.size == 0, f"visibility differs on {bad_vis.size} unambiguous Gaussians, e.g. {bad_vis[:8]}"
    both = na & (vis_g > 0)
    bad_r = np.nonzero(both & (dbg["radius"] != pr.radius))[0]
    assert bad_r.size == 0, f"radius differs on {bad_r.size} Gaussians, e.g. {bad_r[:8]}"
    bad_rect = np.nonzero(both & np.any(dbg["rect"] != pr.rect, axis=1))[0]
    assert bad_rect.size == 0, f"rect differs on {bad_rect.size} Gaussians, e.g. {bad_rect[:8]}"
    # ambiguous: GPU outcome inside the candidate ranges
    c = pr.cand
    a = np.nonzero(amb)[0]
    ok_vis = (vis_g[a] >= c[a, 0]) & (vis_g[a] <= c[a, 1])
    assert np.all(ok_vis), f"ambiguous visibility outside candidates: {a[~ok_vis][:8]}"
    av = a[vis_g[a] > 0]
    ok_r = (dbg["radius"][av] >= c[av, 2]) & (dbg["radius"][av] <= c[av, 3])
    assert np.all(ok_r), f"ambiguous radius outside candidates: {av[~ok_r][:8]}"
    for k in range(4):
        x = dbg["rect"][av, k]
        ok = (x >= c[av, 4 + 2 * k]) & (x <= c[av, 5 + 2 * k])
        assert np.all(ok), f"ambiguous rect edge {k} outside candidates: {av[~ok][:8]}"
    flips = int(np.sum(amb & (vis_g != vis_o)) + np.sum(amb & (vis_g > 0) & (vis_o > 0) &
                                                        ((dbg["radius"] != pr.radius) |
                                                         np.any(dbg["rect"] != pr.rect, axis=1))))
    return {"ambiguous": int(amb.sum()), "ambiguous_flipped": flips}


def compare_list(g: np.ndarray, o: np.ndarray, pr: oracle.Projected) -> int:
    """Compare one tile's GPU list with the oracle's; returns near-tie swaps."""
    amb = pr.amb > 0
    g_na = g[~amb[g]]
    o_na = o[~amb[o]]
    assert g_na.size == o_na.size, f"list lengths differ off ambiguity: {g_na.size} vs {o_na.size}"
    if np.array_equal(g_na, o_na):
        return 0
    assert np.array_equal(np.sort(g_na), np.sort(o_na)), "tile lists differ as multisets"
    z = pr.uvz[:, 2]
    diff = g_na != o_na
    assert np.all(np.abs(z[g_na[diff]] - z[o_na[diff]]) <= DEPTH_TIE_REL * z[o_na[diff]]), "order differs beyond ties"
    return int(diff.sum())


def check_tile_lists(dbg: dict, pr: oracle.Projected, tiles=None) -> dict:
    """All tiles (oracle tile_lists) or the given (tx, ty) tiles (oracle tile_list)."""
    TX, TY = pr.tiles_xy
    gr = dbg["ranges"].astype(np.int64)
    gv = dbg["values"].astype(np.int64)
    # ranges are consistent: contiguous, in tile order, covering all pairs
    assert _ranges_cover(gr, dbg["pairs"]), "GPU tile ranges are not contiguous over the pair array"
    assert int((gr[:, 1] - gr[:, 0]).sum()) == dbg["pairs"]
    swaps = 0
    if tiles is None:
        orr, ov = oracle.tile_lists(pr)
        for t in range(TX * TY):
            swaps += compare_list(gv[gr[t, 0]:gr[t, 1]], ov[orr[t, 0]:orr[t, 1]].astype(np.int64), pr)
        exact_ranges = bool(np.array_equal(gr, orr))
    else:
        for tx, ty in tiles:
            t = ty * TX + tx
            swaps += compare_list(gv[gr[t, 0]:gr[t, 1]], oracle.tile_list(pr, tx, ty).astype(np.int64), pr)
        exact_ranges = None
    return {"near_tie_swaps": swaps, "ranges_exact": exact_ranges}


def _ranges_cover(gr: np.ndarray, P: int) -> bool:
    nz = gr[gr[:, 1] > gr[:, 0]]
    if nz.size == 0:
        return P == 0
    return nz[0, 0] == 0 and nz[-1, 1] == P and np.all(nz[1:, 0] == nz[:-1, 1])


def colour_stats(gpu: np.ndarray, ref: np.ndarray) -> dict:
    d = np.abs(gpu.astype(np.float64) - ref.astype(np.float64))
    per_pixel = d.reshape(-1, d.shape[-1]).max(axis=1)
    return {"max_abs": float(d.max()), "mean_abs": float(d.mean()),
            "frac_within": float(np.mean(per_pixel <= COLOUR_MAX_ABS)),
            "psnr_rgb": oracle.psnr(gpu[..., :3], ref[..., :3])}


def assert_colour(gpu: np.ndarray, ref: np.ndarray) -> dict:
    s = colour_stats(gpu, ref)
    assert s["frac_within"] >= COLOUR_FRACTION, s
    assert s["mean_abs"] <= COLOUR_MEAN_ABS, s
    assert s["psnr_rgb"] >= PSNR_MIN_DB, s
    return s


def encode_rgba8_fp32(f: np.ndarray) -> np.ndarray:
    """The kernels' 8-bit encoding of a float32 frame, reproduced exactly:
    floor(fma(clamp(x, 0, 1), 255, 0.5)) with the fused product-sum rounded
    once to float32.  In float64 the product-sum is exact for every float32 x
    whose rounding can matter (x 255 + 0.5 needs at most 33 significant bits
    there), so rounding it to float32 reproduces the fused operation."""
    c = np.clip(f.astype(np.float32), np.float32(0.0), np.float32(1.0)).astype(np.float64)
    return np.floor((c * 255.0 + 0.5).astype(np.float32)).astype(np.uint8)

