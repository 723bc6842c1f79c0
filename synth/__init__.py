"""Seeded synthetic inputs: scenes, camera poses, trajectories, ABR levels.

This module holds no rasterization arithmetic.  It produces the raw inputs
that both the FP64 oracle (``oracle/``) and the CUDA path read, so that
neither side depends on the other.  Random numbers come from Philox4x32-10
(Salmon et al., SC'11) written in ``synth.c``; every value is addressed by a
counter, so results do not depend on thread count.

Workload shapes follow the paper's setting: scenes of millions of
anisotropic 3D Gaussians (Sec. 1) with the per-Gaussian attributes of
Sec. 5.1 (means, log-scales, quaternions, opacity logits, SH [N][16][3]),
6DoF poses given as azimuth/elevation plus a camera centre (Sec. 5.1 and
the POST /render body of Sec. 5.3), and resolutions chosen from an ABR
ladder (Table 1; the scaled 1920x1080 ladder is used here).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "_synth.so")
_lock = threading.Lock()
_lib = None

BASE_SEED = 20260001


def build(force: bool = False) -> str:
    """Compile ``synth.c`` into ``_synth.so`` (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            dp = ctypes.POINTER(ctypes.c_double)
            fp = ctypes.POINTER(ctypes.c_float)
            lib.synth_philox4x32_10.argtypes = [u32p, u32p, u32p]
            lib.synth_philox4x32_10.restype = None
            lib.synth_normals.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, dp]
            lib.synth_normals.restype = None
            lib.synth_uniforms.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, dp]
            lib.synth_uniforms.restype = None
            lib.synth_scene.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.c_double,
                                        fp, fp, fp, fp, fp]
            lib.synth_scene.restype = ctypes.c_int64
            _lib = lib
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def philox4x32_10(ctr, key) -> tuple[int, int, int, int]:
    """One Philox4x32-10 block: 4-word counter, 2-word key -> 4 words."""
    lib = _load()
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib.synth_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32), _ptr(o, ctypes.c_uint32))
    return tuple(int(x) for x in o)


def normals(seed: int, stream: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    _load().synth_normals(seed, stream, n, _ptr(out, ctypes.c_double))
    return out


def uniforms(seed: int, stream: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    _load().synth_uniforms(seed, stream, n, _ptr(out, ctypes.c_double))
    return out


@dataclass
class Scene:
    """Raw (pre-activation) Gaussian attributes, float32, as a PLY would hold them."""
    means: np.ndarray           # [N,3]
    log_scales: np.ndarray      # [N,3]
    quats: np.ndarray           # [N,4] (w,x,y,z), not normalised
    opacity_logits: np.ndarray  # [N]
    sh: np.ndarray              # [N,16,3]
    sh_degree: int = 3
    seed: int = 0

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "Scene":
        idx = np.asarray(idx)
        return Scene(self.means[idx].copy(), self.log_scales[idx].copy(), self.quats[idx].copy(),
                     self.opacity_logits[idx].copy(), self.sh[idx].copy(), self.sh_degree, self.seed)


def make_scene(n: int, seed: int, n_blobs: int = 64, iso_sigma: float = 0.0, sh_degree: int = 3) -> Scene:
    """Blob-mixture scene (isotropic blobs if ``iso_sigma`` > 0, else anisotropic)."""
    lib = _load()
    means = np.empty((n, 3), np.float32)
    ls = np.empty((n, 3), np.float32)
    q = np.empty((n, 4), np.float32)
    op = np.empty((n,), np.float32)
    sh = np.empty((n, 16, 3), np.float32)
    if n > 0:
        lib.synth_scene(seed, n, n_blobs, iso_sigma, _ptr(means, ctypes.c_float), _ptr(ls, ctypes.c_float),
                        _ptr(q, ctypes.c_float), _ptr(op, ctypes.c_float), _ptr(sh, ctypes.c_float))
    if sh_degree < 3:
        sh[:, (sh_degree + 1) ** 2:, :] = 0.0
    return Scene(means, ls, q, op, sh, sh_degree, seed)


def config_scene(k: int, n: int | None = None) -> Scene:
    """Scene of workload k (1: 100k isotropic blobs; 2..5: anisotropic blobs)."""
    seed = BASE_SEED + k
    if k == 1:
        return make_scene(n or 100_000, seed, n_blobs=8, iso_sigma=0.3)
    sizes = {2: 1_000_000, 3: 3_000_000, 4: 3_000_000, 5: 3_000_000}
    return make_scene(n or sizes[k], seed, n_blobs=64, iso_sigma=0.0)


# ----------------------------------------------------------------- cameras


@dataclass
class Pose:
    """Client pose of the POST /render body: azimuth, elevation (radians), camera centre."""
    azimuth: float
    elevation: float
    t: tuple[float, float, float]


@dataclass
class Intrinsics:
    fx: float
    fy: float
    cx: float
    cy: float


def default_intrinsics(width: int, height: int, vfov_deg: float = 60.0) -> Intrinsics:
    """Pinhole with the given vertical FOV; principal point at the image centre."""
    fy = height / (2.0 * math.tan(math.radians(vfov_deg) / 2.0))
    return Intrinsics(fy, fy, width / 2.0, height / 2.0)


def scale_intrinsics(k: Intrinsics, sx: float, sy: float) -> Intrinsics:
    """Proportional rescale on a resolution change (keeps the FoV, Sec. 6.1)."""
    return Intrinsics(k.fx * sx, k.fy * sy, k.cx * sx, k.cy * sy)


BASE_POSE = Pose(0.0, 0.0, (0.0, 0.0, -3.0))

#: ABR resolution ladder: f x 1920x1080 for f in {0.25, 0.4, 0.5, 2/3, 0.8, 1}
ABR_LEVELS = [(480, 270), (768, 432), (960, 540), (1280, 720), (1536, 864), (1920, 1080)]

#: Table 1 of the paper: (profile, width, height, JPEG quality %, size KB lo, hi)
TABLE1_LADDER = [(3, 320, 180, 10, 6, 8), (2, 640, 360, 35, 18, 22),
                 (1, 960, 540, 65, 50, 60), (0, 1280, 720, 90, 180, 300)]


def trajectory(seed: int, n_poses: int = 300, start: Pose = BASE_POSE, step_t: float = 0.01,
               step_ang_deg: float = 0.5, max_elev_deg: float = 80.0) -> list[Pose]:
    """Random-walk 6DoF trajectory (90 Hz samples): N(0, step_t) per axis on the
    camera centre, N(0, step_ang) on azimuth and elevation, elevation clamped."""
    z = normals(seed, 7, 5 * n_poses).reshape(n_poses, 5)
    poses = []
    az, el = start.azimuth, start.elevation
    t = np.array(start.t, dtype=np.float64)
    lim = math.radians(max_elev_deg)
    for i in range(n_poses):
        if i > 0:
            t = t + step_t * z[i, 0:3]
            az = az + math.radians(step_ang_deg) * z[i, 3]
            el = min(lim, max(-lim, el + math.radians(step_ang_deg) * z[i, 4]))
        poses.append(Pose(float(az), float(el), (float(t[0]), float(t[1]), float(t[2]))))
    return poses


def config_trajectory(k: int, i: int = 0, n_poses: int = 300) -> list[Pose]:
    return trajectory(BASE_SEED + 100 + k + 1000 * i, n_poses)


@dataclass
class ServingTrace:
    """Open-loop request trace of a multi-client serving run, sorted by arrival.

    Per request: arrival time (s), client, scene index, index into the
    client's pose trajectory (90 Hz samples), and the client's link bandwidth
    (bytes/s) in the one-second regime the request falls in."""
    t: np.ndarray            # float64 [R]
    client: np.ndarray       # int32 [R]
    scene: np.ndarray        # int32 [R]
    pose_index: np.ndarray   # int32 [R]
    bw: np.ndarray           # float64 [R], bytes/s
    rates_hz: np.ndarray     # float64 [C]
    seconds: float
    n_scenes: int


def serving_trace(seed: int = BASE_SEED + 500, n_clients: int = 64, seconds: float = 10.0,
                  rate_lo: float = 60.0, rate_hi: float = 90.0, n_scenes: int = 4,
                  bw_median_mbit: float = 22.4, bw_log_sigma: float = 0.75,
                  bw_lo_mbit: float = 5.0, bw_hi_mbit: float = 100.0) -> ServingTrace:
    """Clients with a fixed request rate ~ U[rate_lo, rate_hi] Hz and Poisson
    arrivals; client c renders scene c mod n_scenes (round robin); each client's
    bandwidth is redrawn every second with ln(bw) ~ N(ln median, sigma),
    clipped to [lo, hi] Mbit/s."""
    rates = rate_lo + (rate_hi - rate_lo) * uniforms(seed, 11, n_clients)
    n_sec = int(math.ceil(seconds))
    z = normals(seed, 12, n_clients * n_sec).reshape(n_clients, n_sec)
    bw_mbit = np.clip(np.exp(math.log(bw_median_mbit) + bw_log_sigma * z), bw_lo_mbit, bw_hi_mbit)
    ts, cs, ps, bs = [], [], [], []
    for c in range(n_clients):
        m = int(rates[c] * seconds * 1.5) + 64
        u = uniforms(seed + 1 + c, 13, m)
        arr = np.cumsum(-np.log1p(-u) / rates[c])
        arr = arr[arr < seconds]
        ts.append(arr)
        cs.append(np.full(arr.size, c, np.int32))
        ps.append(np.floor(arr * 90.0).astype(np.int32))
        bs.append(bw_mbit[c, np.minimum(np.floor(arr).astype(np.int64), n_sec - 1)] * 1e6 / 8.0)
    t = np.concatenate(ts)
    o = np.argsort(t, kind="stable")
    client = np.concatenate(cs)[o]
    return ServingTrace(t=t[o], client=client, scene=(client % n_scenes).astype(np.int32),
                        pose_index=np.concatenate(ps)[o], bw=np.concatenate(bs)[o], rates_hz=rates,
                        seconds=float(seconds), n_scenes=n_scenes)


@dataclass
class PoseLogRecord:
    """One logged frame request of a client session: frame index, pose, the
    intrinsics sent with it (at the requested resolution) and the profile."""
    i: int
    pose: Pose
    intr: Intrinsics
    width: int
    height: int
    quality: int


def pose_log(seed: int = BASE_SEED + 600, n_frames: int = 120, ladder=TABLE1_LADDER,
             hold: int = 3) -> list[PoseLogRecord]:
    """A session log: a 90 Hz random-walk trajectory; the profile moves one
    ladder step up or down (or stays) every ``hold`` frames, uniformly."""
    poses = trajectory(seed, n_frames)
    u = uniforms(seed, 31, n_frames)
    levels = sorted(ladder, key=lambda r: r[1])          # low to high resolution
    k = len(levels) - 1
    out = []
    for i in range(n_frames):
        if i > 0 and i % hold == 0:
            k = min(len(levels) - 1, max(0, k + (-1 if u[i] < 1 / 3 else (1 if u[i] > 2 / 3 else 0))))
        _, w, h, q = levels[k][:4]
        out.append(PoseLogRecord(i, poses[i], default_intrinsics(w, h), w, h, q))
    return out
