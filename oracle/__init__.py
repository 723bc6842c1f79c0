"""FP64 CPU oracle for the forward 3DGS rasterization (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg import this package.  The product path (the CUDA library and its Python
binding) never does, and the two share no code: the oracle is ``oracle.c``,
plain C in double precision, compiled here with gcc.

Each function states the part of the paper it follows; the C source gives
the per-step citations (Sec. 5.1 activations, camera and projection
equations; the cited 3DGS rasterizer of Sec. 4.1 for EWA projection, SH
colour and compositing).

Parity status: every function is pinned by tests in ``tests/test_oracle*.py``
(closed forms, invariants, brute force, library special cases); none is
"parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_oracle.so")
_lock = threading.Lock()
_lib = None

TILE = 16

#: default guard bands (relative) around integer decisions: depth, opacity,
#: 3 sqrt(lambda), pixel position.  Within a band the GPU may take any outcome
#: the oracle lists as reachable; off the bands it must match exactly.
DEFAULT_GUARDS = (2.0 ** -16, 2.0 ** -16, 2.0 ** -16, 2.0 ** -18)


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` (gcc -O2 -fopenmp, strict IEEE double: no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            i64, i32, d = ctypes.c_int64, ctypes.c_int, ctypes.c_double
            lib.oracle_camera_rotation.argtypes = [d, d, P]
            lib.oracle_world_to_camera.argtypes = [d, d, P, P]
            lib.oracle_round_half.argtypes = [d]
            lib.oracle_round_half.restype = d
            lib.oracle_sh_basis.argtypes = [i32, P, P]
            lib.oracle_preprocess.argtypes = [i64, P, P, P, P, P, i32, i32, P, i32, i32, P,
                                              P, P, P, P, P, P, P, P, P, P, P]
            lib.oracle_render.argtypes = [i64, P, P, P, P, P, P, i32, i32, P, i64, P, P, P]
            lib.oracle_render_brute.argtypes = [i64, P, P, P, P, P, P, i32, i32, P, i32, P]
            lib.oracle_pair_count.argtypes = [i64, P, P]
            lib.oracle_pair_count.restype = i64
            lib.oracle_tile_lists.argtypes = [i64, P, P, P, i32, i32, P, P]
            lib.oracle_tile_list_one.argtypes = [i64, P, P, P, i32, i32, i64, P]
            lib.oracle_tile_list_one.restype = i64
            lib.oracle_to_rgba8.argtypes = [i64, P, P]
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


# ------------------------------------------------------------------ camera


def camera_rotation(azimuth: float, elevation: float) -> np.ndarray:
    """R = R_y(azimuth) R_x(elevation); columns = camera right/down/forward."""
    R = np.zeros(9)
    _load().oracle_camera_rotation(azimuth, elevation, _p(R))
    return R.reshape(3, 3)


def world_to_camera(azimuth: float, elevation: float, t) -> np.ndarray:
    """T_{w->c} = [R^T, -R^T t; 0, 1] (Sec. 5.1, Rendering Engine)."""
    T = np.zeros(16)
    tt = np.ascontiguousarray(t, dtype=np.float64)
    _load().oracle_world_to_camera(azimuth, elevation, _p(tt), _p(T))
    return T.reshape(4, 4)


def round_half(x: float) -> float:
    """Nearest IEEE binary16 value (ties to even)."""
    return _load().oracle_round_half(float(x))


def sh_basis(direction, degree: int = 3) -> np.ndarray:
    """Real SH basis values Y_0..Y_15 at a unit direction (Legendre form)."""
    d = np.ascontiguousarray(direction, dtype=np.float64)
    Y = np.zeros(16)
    _load().oracle_sh_basis(degree, _p(d), _p(Y))
    return Y


# -------------------------------------------------------------- preprocess


@dataclass
class Projected:
    visible: np.ndarray  # int8 [N]
    cull: np.ndarray     # int8 [N]
    uvz: np.ndarray      # f64 [N,3]
    conic: np.ndarray    # f64 [N,3]
    opacity: np.ndarray  # f64 [N]
    rgb: np.ndarray      # f64 [N,3]
    radius: np.ndarray   # i32 [N]
    rect: np.ndarray     # i32 [N,4]
    cand: np.ndarray     # i32 [N,12]
    amb: np.ndarray      # int8 [N]
    dq: np.ndarray       # f64 [N,4]
    width: int
    height: int

    @property
    def tiles_touched(self) -> np.ndarray:
        r = self.rect.astype(np.int64)
        t = (r[:, 2] - r[:, 0]) * (r[:, 3] - r[:, 1])
        return np.where(self.visible > 0, t, 0)

    @property
    def tiles_xy(self) -> tuple[int, int]:
        return (self.width + TILE - 1) // TILE, (self.height + TILE - 1) // TILE


def camera_vector(pose, intr) -> np.ndarray:
    return np.array([pose.azimuth, pose.elevation, pose.t[0], pose.t[1], pose.t[2],
                     intr.fx, intr.fy, intr.cx, intr.cy], dtype=np.float64)


def preprocess(scene, pose, intr, width: int, height: int, storage_half: bool = False,
               guards=DEFAULT_GUARDS) -> Projected:
    """FP64 per-Gaussian projection, culling, conic, radius, rect and colour."""
    lib = _load()
    n = scene.n
    means, ls, q = _f32(scene.means), _f32(scene.log_scales), _f32(scene.quats)
    op, sh = _f32(scene.opacity_logits), _f32(scene.sh)
    cam = camera_vector(pose, intr)
    g = np.ascontiguousarray(guards, dtype=np.float64)
    out = Projected(np.zeros(n, np.int8), np.zeros(n, np.int8), np.zeros((n, 3)), np.zeros((n, 3)),
                    np.zeros(n), np.zeros((n, 3)), np.zeros(n, np.int32), np.zeros((n, 4), np.int32),
                    np.zeros((n, 12), np.int32), np.zeros(n, np.int8), np.zeros((n, 4)), width, height)
    lib.oracle_preprocess(n, _p(means), _p(ls), _p(q), _p(op), _p(sh), int(scene.sh_degree),
                          int(storage_half), _p(cam), width, height, _p(g),
                          _p(out.visible), _p(out.cull), _p(out.uvz), _p(out.conic), _p(out.opacity),
                          _p(out.rgb), _p(out.radius), _p(out.rect), _p(out.cand), _p(out.amb), _p(out.dq))
    return out


# --------------------------------------------------------------- compositing


def render(pr: Projected, background=(0.0, 0.0, 0.0), pixels=None, want_evals: bool = False):
    """Float RGBA (alpha = 1 - T) of the whole frame [H,W,4] or of the given
    (x, y) pixels [n,4]; optionally the per-pixel count of list entries visited."""
    lib = _load()
    bg = np.ascontiguousarray(background, dtype=np.float64)
    W, H = pr.width, pr.height
    if pixels is None:
        out = np.zeros((H * W, 4))
        npix, pp = H * W, None
    else:
        pix = np.ascontiguousarray(pixels, dtype=np.int32).reshape(-1, 2)
        out = np.zeros((pix.shape[0], 4))
        npix, pp = pix.shape[0], _p(pix)
    ev = np.zeros(npix, np.int64) if want_evals else None
    lib.oracle_render(pr.visible.shape[0], _p(pr.visible), _p(pr.uvz), _p(pr.conic), _p(pr.opacity),
                      _p(pr.rgb), _p(pr.rect), W, H, _p(bg), npix, pp, _p(out),
                      _p(ev) if ev is not None else None)
    if pixels is None:
        out = out.reshape(H, W, 4)
        if ev is not None:
            ev = ev.reshape(H, W)
    return (out, ev) if want_evals else out


def render_brute(pr: Projected, background=(0.0, 0.0, 0.0), support_rule: bool = True) -> np.ndarray:
    """Per-pixel brute force over every Gaussian (tiny scenes only)."""
    lib = _load()
    bg = np.ascontiguousarray(background, dtype=np.float64)
    out = np.zeros((pr.height * pr.width, 4))
    lib.oracle_render_brute(pr.visible.shape[0], _p(pr.visible), _p(pr.uvz), _p(pr.conic),
                            _p(pr.opacity), _p(pr.rgb), _p(pr.rect), pr.width, pr.height, _p(bg),
                            int(support_rule), _p(out))
    return out.reshape(pr.height, pr.width, 4)


def to_rgba8(rgba: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(rgba, dtype=np.float64)
    out = np.zeros(a.shape, np.uint8)
    _load().oracle_to_rgba8(a.size // 4, _p(a), _p(out))
    return out


# ---------------------------------------------------------------- tile lists


def pair_count(pr: Projected) -> int:
    return int(_load().oracle_pair_count(pr.visible.shape[0], _p(pr.visible), _p(pr.rect)))


def tile_lists(pr: Projected) -> tuple[np.ndarray, np.ndarray]:
    """Per-tile (depth, index)-ordered lists: ranges [T,2] (int64) and values [P]."""
    lib = _load()
    TX, TY = pr.tiles_xy
    P = pair_count(pr)
    ranges = np.zeros((TX * TY, 2), np.int64)
    values = np.zeros(max(P, 1), np.int32)
    lib.oracle_tile_lists(pr.visible.shape[0], _p(pr.visible), _p(pr.uvz), _p(pr.rect),
                          pr.width, pr.height, _p(ranges), _p(values))
    return ranges, values[:P]


def tile_list(pr: Projected, tx: int, ty: int) -> np.ndarray:
    lib = _load()
    n = pr.visible.shape[0]
    length = lib.oracle_tile_list_one(n, _p(pr.visible), _p(pr.uvz), _p(pr.rect), tx, ty, 0, None)
    out = np.zeros(max(length, 1), np.int32)
    lib.oracle_tile_list_one(n, _p(pr.visible), _p(pr.uvz), _p(pr.rect), tx, ty, length, _p(out))
    return out[:length]


def psnr(a: np.ndarray, b: np.ndarray) -> float:
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return float("inf") if mse == 0 else 10.0 * np.log10(1.0 / mse)
