"""Deterministic post-session replay (Sec. 5.3, "Sampled OPFS Capture and
Post-Session Materialization").

A client session is logged as one record per frame request: frame index,
pose, the intrinsics sent with the request and the ABR profile (resolution
and JPEG quality).  After the session the backend replays the records at the
sampled indices and materializes, per sampled frame, (i) the transmitted
JPEG -- the frame rendered at the profile's resolution and encoded at its
quality, byte-identical to what was sent -- and (ii) a lossless ground-truth
PNG rendered at the display resolution, with the intrinsics scaled to it
(field of view unchanged).  Every render and encode is deterministic, so a
replay reproduces the same bytes.

Each sampled frame also gets SSIM and PSNR, computed on the GPU, between the
ground truth and the transmitted-resolution render upsampled bilinearly to
the display resolution (the resolution loss of the chosen profile; the JPEG
loss itself is not decoded here).
"""
from __future__ import annotations

import json
import os
import struct
import zlib
from dataclasses import dataclass

import numpy as np

from . import tigas as tb


@dataclass
class ReplayFrame:
    i: int
    width: int
    height: int
    quality: int
    jpeg: bytes
    gt: np.ndarray | None      # [H, W, 4] uint8 (host) when kept
    ssim: float
    psnr: float


def write_pose_log(path, records, display: tuple[int, int]) -> None:
    """JSON lines: a header {"display": [W, H]} then one object per record."""
    with open(path, "w") as f:
        f.write(json.dumps({"display": list(display)}) + "\n")
        for r in records:
            p, k = tb.make_pose(r.pose), tb.make_intrinsics(r.intr)
            f.write(json.dumps({"i": r.i, "pose": [p.azimuth, p.elevation, list(p.t)],
                                "intr": [k.fx, k.fy, k.cx, k.cy], "width": r.width, "height": r.height,
                                "quality": r.quality}) + "\n")


@dataclass
class LogRecord:
    i: int
    pose: tuple
    intr: tuple
    width: int
    height: int
    quality: int


def read_pose_log(path) -> tuple[list[LogRecord], tuple[int, int]]:
    with open(path) as f:
        head = json.loads(f.readline())
        recs = []
        for line in f:
            if line.strip():
                d = json.loads(line)
                az, el, t = d["pose"]
                recs.append(LogRecord(int(d["i"]), (az, el, tuple(t)), tuple(d["intr"]), int(d["width"]),
                                      int(d["height"]), int(d["quality"])))
    return recs, tuple(head["display"])


def png_bytes(rgba: np.ndarray) -> bytes:
    """A PNG (colour type 6, 8 bits, no filtering, zlib level 6) of an RGBA8 frame."""
    h, w = rgba.shape[:2]

    def chunk(tag: bytes, data: bytes) -> bytes:
        return struct.pack(">I", len(data)) + tag + data + struct.pack(">I", zlib.crc32(tag + data) & 0xFFFFFFFF)

    raw = np.concatenate([np.zeros((h, 1), np.uint8), np.ascontiguousarray(rgba).reshape(h, w * 4)], axis=1)
    return (b"\x89PNG\r\n\x1a\n" + chunk(b"IHDR", struct.pack(">IIBBBBB", w, h, 8, 6, 0, 0, 0)) +
            chunk(b"IDAT", zlib.compress(raw.tobytes(), 6)) + chunk(b"IEND", b""))


def _scaled(intr, sx: float, sy: float):
    k = tb.make_intrinsics(intr)
    return tb.Intrinsics(k.fx * sx, k.fy * sy, k.cx * sx, k.cy * sy)


def replay(scene, records, display: tuple[int, int], stride: int = 1, out_dir=None, restart_mcus: int = 2,
           keep_gt: bool = False, batch: int = 8) -> list[ReplayFrame]:
    """Replay the records whose index is a multiple of ``stride``.  With
    out_dir, writes <i>_original.jpg and <i>_gt.png per sampled frame."""
    import torch

    W, H = display
    dev = torch.device("cuda")
    picked = [r for r in records if r.i % stride == 0]
    out: list[ReplayFrame] = []
    if out_dir is not None:
        os.makedirs(out_dir, exist_ok=True)
    for s in range(0, len(picked), batch):
        grp = picked[s:s + batch]
        low = [torch.empty((r.height, r.width, 4), dtype=torch.uint8, device=dev) for r in grp]
        gt = [torch.empty((H, W, 4), dtype=torch.uint8, device=dev) for _ in grp]
        tb.render_batch(scene, [r.pose for r in grp], [r.intr for r in grp], [r.width for r in grp],
                        [r.height for r in grp], low)
        tb.render_batch(scene, [r.pose for r in grp], [_scaled(r.intr, W / r.width, H / r.height) for r in grp],
                        [W] * len(grp), [H] * len(grp), gt)
        up = torch.empty((H, W, 4), dtype=torch.uint8, device=dev)
        for r, lo, g in zip(grp, low, gt):
            jpg = tb.jpeg_encode(lo, r.quality, restart_mcus=restart_mcus)
            tb.resample_rgba8(lo, W, H, out=up)
            q = tb.image_quality(g, up)
            g_host = g.cpu().numpy() if (keep_gt or out_dir is not None) else None
            if out_dir is not None:
                with open(os.path.join(out_dir, f"{r.i:06d}_original.jpg"), "wb") as f:
                    f.write(jpg)
                with open(os.path.join(out_dir, f"{r.i:06d}_gt.png"), "wb") as f:
                    f.write(png_bytes(g_host))
            out.append(ReplayFrame(r.i, r.width, r.height, r.quality, jpg, g_host if keep_gt else None,
                                   q["ssim"], q["psnr"]))
    return out
