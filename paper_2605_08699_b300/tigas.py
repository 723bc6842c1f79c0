"""ctypes binding of ``libtigas.so`` (declared in ``include/tigas.h``).

Argument marshalling only: every step of the render path runs in the CUDA
library.  Arrays may be numpy arrays (host memory) or torch tensors (host or
device; only their data pointers and streams are used).  There is no CPU
fallback: if the library is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Any, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtigas.so")

OK, ERR_INVALID, ERR_OOM, ERR_CUDA, ERR_AGAIN, ERR_OVERFLOW, ERR_TIMEOUT, ERR_NOT_FOUND, ERR_IO = range(9)
STORAGE_FP32, STORAGE_FP16 = 0, 1
SORT_DEPTH_FIRST, SORT_FULL64, SORT_SLICED = 0, 1, 2

#: every symbol include/tigas.h declares
EXPORTS = ["tigas_scene_load", "tigas_scene_free", "tigas_scene_bytes", "tigas_render", "tigas_render_ex",
           "tigas_render_batch", "tigas_debug_render", "tigas_sort_pairs_u64", "tigas_server_create",
           "tigas_server_destroy", "tigas_server_submit", "tigas_server_poll", "tigas_last_error",
           "tigas_version", "tigas_kernel_launches", "tigas_profile_enable", "tigas_profile_read",
           "tigas_sort_pairs_u64_noalloc", "tigas_sort_noalloc_check", "tigas_debug_sort_noalloc_wait_timeout",
           "tigas_render_batch_ex", "tigas_set_graphs", "tigas_debug_sort_wait_timeout",
           "tigas_set_schedule", "tigas_set_schedule_for_views", "tigas_get_schedule", "tigas_autotune", "tigas_exact_rerenders",
           "tigas_jpeg_encode", "tigas_ply_probe", "tigas_ply_decode", "tigas_scene_load_ply",
           "tigas_registry_open", "tigas_registry_scan", "tigas_registry_count", "tigas_registry_info",
           "tigas_registry_acquire", "tigas_registry_release", "tigas_registry_evict_idle",
           "tigas_registry_start_eviction", "tigas_registry_set_clock", "tigas_registry_close",
           "tigas_resample_rgba8", "tigas_image_quality", "tigas_profile_stages", "tigas_render_batch_async",
           "tigas_render_wait", "tigas_debug_fail_alloc", "tigas_release_workspace"]

STAGES = ["preprocess", "depth_sort", "scan", "emit", "pair_sort", "ranges", "blend", "frame"]


class TigasError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"tigas status {status}: {message}")
        self.status = status


class Pose(ctypes.Structure):
    _fields_ = [("azimuth", ctypes.c_double), ("elevation", ctypes.c_double), ("t", ctypes.c_double * 3)]


class Intrinsics(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_double), ("fy", ctypes.c_double), ("cx", ctypes.c_double), ("cy", ctypes.c_double)]


class SceneDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("sh_degree", ctypes.c_int), ("storage", ctypes.c_int),
                ("means", ctypes.c_void_p), ("log_scales", ctypes.c_void_p), ("quats", ctypes.c_void_p),
                ("opacity_logits", ctypes.c_void_p), ("sh", ctypes.c_void_p), ("inputs_on_device", ctypes.c_int),
                ("background", ctypes.c_float * 3)]


class FrameStats(ctypes.Structure):
    _fields_ = [("n_visible", ctypes.c_uint64), ("n_pairs", ctypes.c_uint64), ("n_tiles", ctypes.c_uint32),
                ("sort_passes", ctypes.c_uint32), ("blend_evals", ctypes.c_uint64), ("blend_fetched", ctypes.c_uint64),
                ("blend_contribs", ctypes.c_uint64), ("depth_sort_passes", ctypes.c_uint32),
                ("depth_sort_near", ctypes.c_uint32)]


class DebugFrame(ctypes.Structure):
    _fields_ = [("visible", ctypes.c_void_p), ("radius", ctypes.c_void_p), ("rect", ctypes.c_void_p),
                ("depth", ctypes.c_void_p), ("uv", ctypes.c_void_p), ("q", ctypes.c_void_p),
                ("values", ctypes.c_void_p), ("pair_capacity", ctypes.c_uint64), ("ranges", ctypes.c_void_p),
                ("rgba_f32", ctypes.c_void_p)]


class Schedule(ctypes.Structure):
    _fields_ = [("n_slices", ctypes.c_int), ("first_slice_inv", ctypes.c_int), ("blend_ctas_per_sm", ctypes.c_int),
                ("blend_batch", ctypes.c_int), ("views_per_set", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {"n_slices": self.n_slices, "first_slice_inv": self.first_slice_inv,
                "blend_ctas_per_sm": self.blend_ctas_per_sm, "blend_batch": self.blend_batch,
                "views_per_set": self.views_per_set}


class ServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_uint64), ("max_batch", ctypes.c_int), ("max_inflight", ctypes.c_int),
                ("batch_window_us", ctypes.c_int)]


class Completion(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("client_id", ctypes.c_uint64), ("status", ctypes.c_int),
                ("width", ctypes.c_int), ("height", ctypes.c_int), ("submit_us", ctypes.c_double),
                ("admit_us", ctypes.c_double), ("done_us", ctypes.c_double)]


class PlyInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("file_bytes", ctypes.c_uint64), ("body_offset", ctypes.c_uint64),
                ("sh_degree", ctypes.c_int), ("format", ctypes.c_int), ("row_bytes", ctypes.c_uint32),
                ("n_properties", ctypes.c_uint32)]


class ModelInfo(ctypes.Structure):
    _fields_ = [("id", ctypes.c_char * 128), ("name", ctypes.c_char * 128), ("ply_path", ctypes.c_char * 1024),
                ("preview_path", ctypes.c_char * 1024), ("n", ctypes.c_uint64), ("file_bytes", ctypes.c_uint64),
                ("resident_bytes", ctypes.c_uint64), ("loads", ctypes.c_uint64), ("idle_seconds", ctypes.c_double),
                ("sh_degree", ctypes.c_int), ("loaded", ctypes.c_int), ("users", ctypes.c_int),
                ("reserved", ctypes.c_int)]


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libtigas.so (raises when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -m paper_2605_08699_b300.build`")
    lib = ctypes.CDLL(path)
    P, i, st = ctypes.c_void_p, ctypes.c_int, ctypes.c_int
    sig = {
        "tigas_scene_load": (st, [ctypes.POINTER(SceneDesc), ctypes.POINTER(P)]),
        "tigas_scene_free": (st, [P]),
        "tigas_scene_bytes": (st, [P, ctypes.POINTER(ctypes.c_uint64)]),
        "tigas_render": (st, [P, ctypes.POINTER(Pose), ctypes.POINTER(Intrinsics), i, i, P]),
        "tigas_render_ex": (st, [P, ctypes.POINTER(Pose), ctypes.POINTER(Intrinsics), i, i, P, P, P, i,
                                 ctypes.POINTER(FrameStats)]),
        "tigas_render_batch": (st, [P, i, ctypes.POINTER(Pose), ctypes.POINTER(Intrinsics), P, P, P, P]),
        "tigas_render_batch_ex": (st, [P, i, ctypes.POINTER(Pose), ctypes.POINTER(Intrinsics), P, P, P, P, i,
                                       ctypes.POINTER(FrameStats)]),
        "tigas_render_batch_async": (st, [P, i, ctypes.POINTER(Pose), ctypes.POINTER(Intrinsics), P, P, P, P,
                                          ctypes.POINTER(P)]),
        "tigas_render_wait": (st, [P]),
        "tigas_debug_render": (st, [P, ctypes.POINTER(Pose), ctypes.POINTER(Intrinsics), i, i, i,
                                    ctypes.POINTER(DebugFrame), ctypes.POINTER(ctypes.c_uint64)]),
        "tigas_sort_pairs_u64": (st, [P, P, P, P, ctypes.c_uint64, i, i, P]),
        "tigas_sort_pairs_u64_noalloc": (st, [P, P, P, P, ctypes.c_uint64, i, i, P]),
        "tigas_sort_noalloc_check": (st, [P]),
        "tigas_debug_sort_noalloc_wait_timeout": (st, [i, P]),
        "tigas_server_create": (st, [ctypes.POINTER(ServerConfig), ctypes.POINTER(P)]),
        "tigas_server_destroy": (st, [P, i]),
        "tigas_server_submit": (st, [P, P, ctypes.POINTER(Pose), ctypes.POINTER(Intrinsics), i, i, P,
                                     ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)]),
        "tigas_server_poll": (st, [P, ctypes.POINTER(Completion), i, i, ctypes.POINTER(ctypes.c_int)]),
        "tigas_last_error": (ctypes.c_char_p, []),
        "tigas_version": (ctypes.c_char_p, []),
        "tigas_kernel_launches": (ctypes.c_uint64, []),
        "tigas_profile_enable": (st, [i]),
        "tigas_profile_stages": (st, [ctypes.c_uint32]),
        "tigas_set_graphs": (st, [i]),
        "tigas_debug_sort_wait_timeout": (st, [i]),
        "tigas_debug_fail_alloc": (st, [i, ctypes.c_int64, ctypes.c_int64]),
        "tigas_release_workspace": (st, []),
        "tigas_set_schedule": (st, [ctypes.POINTER(Schedule)]),
        "tigas_set_schedule_for_views": (st, [i, ctypes.POINTER(Schedule)]),
        "tigas_get_schedule": (st, [i, ctypes.POINTER(Schedule)]),
        "tigas_exact_rerenders": (ctypes.c_uint64, []),
        "tigas_jpeg_encode": (st, [P, i, i, i, i, P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64), P]),
        "tigas_autotune": (st, [P, i, i, ctypes.POINTER(Pose), ctypes.POINTER(Intrinsics), ctypes.POINTER(ctypes.c_int),
                                ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_void_p), i,
                                ctypes.POINTER(Schedule), ctypes.POINTER(ctypes.c_double)]),
        "tigas_profile_read": (st, [P, P, i]),
        "tigas_ply_probe": (st, [ctypes.c_char_p, ctypes.POINTER(PlyInfo)]),
        "tigas_ply_decode": (st, [ctypes.c_char_p, P, P, P, P, P, i]),
        "tigas_scene_load_ply": (st, [ctypes.c_char_p, i, P, ctypes.POINTER(P)]),
        "tigas_registry_open": (st, [ctypes.c_char_p, i, ctypes.c_double, ctypes.c_uint64, P, ctypes.POINTER(P)]),
        "tigas_registry_scan": (st, [P, ctypes.POINTER(i), ctypes.POINTER(i)]),
        "tigas_registry_count": (st, [P, ctypes.POINTER(i)]),
        "tigas_registry_info": (st, [P, i, ctypes.POINTER(ModelInfo)]),
        "tigas_registry_acquire": (st, [P, ctypes.c_char_p, ctypes.POINTER(P)]),
        "tigas_registry_release": (st, [P, P]),
        "tigas_registry_evict_idle": (st, [P, ctypes.POINTER(i)]),
        "tigas_registry_start_eviction": (st, [P, ctypes.c_double]),
        "tigas_registry_set_clock": (st, [P, ctypes.c_double]),
        "tigas_registry_close": (st, [P]),
        "tigas_resample_rgba8": (st, [P, i, i, P, i, i, P]),
        "tigas_image_quality": (st, [P, P, i, i, P, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double), P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(status: int) -> None:
    if status != OK:
        raise TigasError(status, _lib.tigas_last_error().decode())


def last_error() -> str:
    return load_library().tigas_last_error().decode()


def version() -> str:
    return load_library().tigas_version().decode()


def kernel_launches() -> int:
    return int(load_library().tigas_kernel_launches())


def profile_enable(on: bool = True) -> None:
    """Per-stage CUDA-event timing of every later render (tigas_profile_enable)."""
    _check(load_library().tigas_profile_enable(int(on)))


def profile_stages(stages) -> None:
    """Time only the named stages (tigas_profile_stages); an empty list turns timing off."""
    mask = 0
    for name in stages:
        mask |= 1 << STAGES.index(name)
    _check(load_library().tigas_profile_stages(mask))


def set_graphs(on: bool = True) -> None:
    """Capture and replay CUDA graphs of the sliced schedule (tigas_set_graphs)."""
    _check(load_library().tigas_set_graphs(int(on)))


def debug_sort_wait_timeout(spin_limit: int) -> int:
    """Run the radix sort's look-back timeout hook; returns the tigas status
    (TIMEOUT = 6 is the expected outcome)."""
    return int(load_library().tigas_debug_sort_wait_timeout(int(spin_limit)))


DEVICE_ALLOC, PINNED_ALLOC = 0, 1


def debug_fail_alloc(kind: int, nth: int = 1, count: int = 1) -> None:
    """Make allocations nth .. nth + count - 1 of a kind fail (tigas_debug_fail_alloc);
    nth = 0 clears the kind."""
    _check(load_library().tigas_debug_fail_alloc(int(kind), int(nth), int(count)))


def release_workspace() -> None:
    """Free the workspace of idle render contexts (tigas_release_workspace)."""
    _check(load_library().tigas_release_workspace())


def profile_read(reset: bool = False) -> dict:
    """Accumulated GPU milliseconds and launch-set counts per stage."""
    ms = (ctypes.c_double * len(STAGES))()
    calls = (ctypes.c_uint64 * len(STAGES))()
    _check(load_library().tigas_profile_read(ctypes.cast(ms, ctypes.c_void_p), ctypes.cast(calls, ctypes.c_void_p),
                                             int(reset)))
    return {name: {"ms": ms[k], "calls": int(calls[k])} for k, name in enumerate(STAGES)}


# ------------------------------------------------------------ marshalling


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x) -> int | None:
    if x is None:
        return None
    if _is_torch(x):
        assert x.is_contiguous(), "tensor must be contiguous"
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"], "array must be C-contiguous"
        return x.ctypes.data
    if isinstance(x, int):
        return x
    raise TypeError(f"unsupported buffer type {type(x)}")


def _on_device(x) -> bool:
    return _is_torch(x) and x.is_cuda


def _stream(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)   # torch.cuda.Stream


def make_pose(p) -> Pose:
    if isinstance(p, Pose):
        return p
    if hasattr(p, "azimuth"):
        return Pose(p.azimuth, p.elevation, (ctypes.c_double * 3)(*p.t))
    az, el, t = p
    return Pose(az, el, (ctypes.c_double * 3)(*t))


def make_intrinsics(k) -> Intrinsics:
    if isinstance(k, Intrinsics):
        return k
    if hasattr(k, "fx"):
        return Intrinsics(k.fx, k.fy, k.cx, k.cy)
    return Intrinsics(*k)


# ----------------------------------------------------------------- scenes


class SceneHandle:
    """A resident scene (``tigas_scene*``); free() drops the caller's reference."""

    def __init__(self, handle: int, n: int, storage: int):
        self.handle = handle
        self.n = n
        self.storage = storage

    @property
    def bytes(self) -> int:
        out = ctypes.c_uint64()
        _check(load_library().tigas_scene_bytes(self.handle, ctypes.byref(out)))
        return int(out.value)

    def free(self) -> None:
        if self.handle:
            _check(load_library().tigas_scene_free(self.handle))
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.free()


def scene_load(means, log_scales, quats, opacity_logits, sh, sh_degree: int = 3, storage: int = STORAGE_FP32,
               background=(0.0, 0.0, 0.0)) -> SceneHandle:
    """Upload raw attributes (float32, see tigas_scene_desc) and activate them."""
    arrs = [means, log_scales, quats, opacity_logits, sh]
    dev = [_on_device(a) for a in arrs]
    if any(dev) and not all(dev):
        raise ValueError("attribute arrays must be all host or all device")
    if not dev[0]:
        arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in arrs]
    n = int(arrs[0].shape[0])
    d = SceneDesc(n, sh_degree, storage, *[_ptr(a) for a in arrs], int(dev[0]), (ctypes.c_float * 3)(*background))
    h = ctypes.c_void_p()
    _check(load_library().tigas_scene_load(ctypes.byref(d), ctypes.byref(h)))
    return SceneHandle(h.value, n, storage)


def scene_from(s, storage: int = STORAGE_FP32, background=(0.0, 0.0, 0.0)) -> SceneHandle:
    """Load an object with means/log_scales/quats/opacity_logits/sh/sh_degree attributes."""
    return scene_load(s.means, s.log_scales, s.quats, s.opacity_logits, s.sh, s.sh_degree, storage, background)


# ------------------------------------------------------------ PLY models

PLY_FORMATS = ("binary_little_endian", "binary_big_endian", "ascii")


def _path(p) -> bytes:
    return os.fsencode(os.fspath(p))


def ply_probe(path) -> dict:
    """Header of a 3DGS PLY file (tigas_ply_probe; host only)."""
    info = PlyInfo()
    _check(load_library().tigas_ply_probe(_path(path), ctypes.byref(info)))
    return {"n": int(info.n), "file_bytes": int(info.file_bytes), "body_offset": int(info.body_offset),
            "sh_degree": info.sh_degree, "format": PLY_FORMATS[info.format], "row_bytes": int(info.row_bytes),
            "n_properties": int(info.n_properties)}


def ply_decode(path, out: dict | None = None) -> dict:
    """Raw attribute arrays of a PLY (tigas_ply_decode).  ``out`` may hold
    preallocated float32 arrays (all host numpy or all CUDA tensors) under the
    keys means, log_scales, quats, opacity_logits, sh; else host arrays are made."""
    n = ply_probe(path)["n"]
    if out is None:
        out = {"means": np.empty((n, 3), np.float32), "log_scales": np.empty((n, 3), np.float32),
               "quats": np.empty((n, 4), np.float32), "opacity_logits": np.empty((n,), np.float32),
               "sh": np.empty((n, 16, 3), np.float32)}
    keys = ("means", "log_scales", "quats", "opacity_logits", "sh")
    dev = [_on_device(out[k]) for k in keys]
    if any(dev) and not all(dev):
        raise ValueError("outputs must be all host or all device")
    _check(load_library().tigas_ply_decode(_path(path), *[_ptr(out[k]) for k in keys], int(dev[0])))
    return out


def scene_load_ply(path, storage: int = STORAGE_FP32, background=(0.0, 0.0, 0.0)) -> SceneHandle:
    """Load a 3DGS PLY straight into a resident scene (tigas_scene_load_ply)."""
    bg = (ctypes.c_float * 3)(*background)
    h = ctypes.c_void_p()
    _check(load_library().tigas_scene_load_ply(_path(path), storage, ctypes.cast(bg, ctypes.c_void_p),
                                               ctypes.byref(h)))
    n = ply_probe(path)["n"]
    return SceneHandle(h.value, n, storage)


class RegistryScene(SceneHandle):
    """A scene acquired from a Registry; free() hands it back (tigas_registry_release)."""

    def __init__(self, registry: "Registry", handle: int, model_id: str, n: int, storage: int):
        super().__init__(handle, n, storage)
        self.registry = registry
        self.model_id = model_id

    def free(self) -> None:
        if self.handle:
            if self.registry.handle:
                _check(load_library().tigas_registry_release(self.registry.handle, self.handle))
            else:   # the registry was closed first: drop the reference directly
                _check(load_library().tigas_scene_free(self.handle))
            self.handle = None


class Registry:
    """Model registry over a folder of 3DGS models (tigas_registry_*): lazy
    load on first acquire, shared and reference-counted while acquired,
    unloaded after idle_timeout_s without users."""

    def __init__(self, root, storage: int = STORAGE_FP16, idle_timeout_s: float = 60.0,
                 resident_budget_bytes: int = 0, background=(0.0, 0.0, 0.0)):
        self.storage = storage
        bg = (ctypes.c_float * 3)(*background)
        h = ctypes.c_void_p()
        _check(load_library().tigas_registry_open(_path(root), storage, float(idle_timeout_s),
                                                  int(resident_budget_bytes), ctypes.cast(bg, ctypes.c_void_p),
                                                  ctypes.byref(h)))
        self.handle = h.value

    def scan(self) -> tuple[int, int]:
        n, skipped = ctypes.c_int(), ctypes.c_int()
        _check(load_library().tigas_registry_scan(self.handle, ctypes.byref(n), ctypes.byref(skipped)))
        return n.value, skipped.value

    def __len__(self) -> int:
        n = ctypes.c_int()
        _check(load_library().tigas_registry_count(self.handle, ctypes.byref(n)))
        return n.value

    def info(self, index: int) -> dict:
        m = ModelInfo()
        _check(load_library().tigas_registry_info(self.handle, index, ctypes.byref(m)))
        out = {k: getattr(m, k) for k, _ in ModelInfo._fields_ if k != "reserved"}
        for k in ("id", "name", "ply_path", "preview_path"):
            out[k] = out[k].decode()
        out["loaded"] = bool(out["loaded"])
        return out

    def models(self) -> list[dict]:
        return [self.info(k) for k in range(len(self))]

    def model(self, model_id: str) -> dict:
        for m in self.models():
            if m["id"] == model_id:
                return m
        raise KeyError(model_id)

    def acquire(self, model_id: str) -> RegistryScene:
        h = ctypes.c_void_p()
        _check(load_library().tigas_registry_acquire(self.handle, model_id.encode(), ctypes.byref(h)))
        return RegistryScene(self, h.value, model_id, self.model(model_id)["n"], self.storage)

    def evict_idle(self) -> int:
        k = ctypes.c_int()
        _check(load_library().tigas_registry_evict_idle(self.handle, ctypes.byref(k)))
        return k.value

    def start_eviction(self, period_s: float) -> None:
        _check(load_library().tigas_registry_start_eviction(self.handle, float(period_s)))

    def set_clock(self, now_s: float | None) -> None:
        _check(load_library().tigas_registry_set_clock(self.handle, -1.0 if now_s is None else float(now_s)))

    def close(self) -> None:
        if self.handle:
            _check(load_library().tigas_registry_close(self.handle))
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# -------------------------------------------------------- quality metrics


def resample_rgba8(src, width: int, height: int, out=None, stream=None):
    """Bilinear RGBA8 resample (tigas_resample_rgba8).  src: [h, w, 4] uint8,
    host numpy or CUDA tensor; returns ``out`` (new host array if None)."""
    h, w = int(src.shape[0]), int(src.shape[1])
    if out is None:
        out = np.empty((height, width, 4), np.uint8)
    _check(load_library().tigas_resample_rgba8(_ptr(src), w, h, _ptr(out), width, height, _stream(stream)))
    return out


def image_quality(a, b, ssim_map=None, stream=None) -> dict:
    """SSIM and PSNR of two RGBA8 frames of equal size (tigas_image_quality).
    ssim_map: optional float32 [H-10, W-10] host array or CUDA tensor."""
    if tuple(a.shape) != tuple(b.shape):
        raise ValueError("frames differ in shape")
    h, w = int(a.shape[0]), int(a.shape[1])
    s, p = ctypes.c_double(), ctypes.c_double()
    _check(load_library().tigas_image_quality(_ptr(a), _ptr(b), w, h, _ptr(ssim_map), ctypes.byref(s),
                                              ctypes.byref(p), _stream(stream)))
    return {"ssim": s.value, "psnr": p.value}


# ---------------------------------------------------------------- render


def render(scene: SceneHandle, pose, intr, width: int, height: int, out=None):
    """tigas_render.  Returns ``out`` (a new host [H, W, 4] uint8 array if None)."""
    if out is None:
        out = np.empty((height, width, 4), np.uint8)
    _check(load_library().tigas_render(scene.handle, ctypes.byref(make_pose(pose)),
                                       ctypes.byref(make_intrinsics(intr)), width, height, _ptr(out)))
    return out


def _stats_dict(stats: "FrameStats") -> dict:
    return {"n_visible": stats.n_visible, "n_pairs": stats.n_pairs, "n_tiles": stats.n_tiles,
            "sort_passes": stats.sort_passes, "blend_evals": stats.blend_evals, "blend_fetched": stats.blend_fetched,
            "blend_contribs": stats.blend_contribs, "depth_sort_passes": stats.depth_sort_passes,
            "depth_sort_near": stats.depth_sort_near}


def render_ex(scene: SceneHandle, pose, intr, width: int, height: int, out_rgba8=None, out_rgba_f32=None,
              stream=None, sort_mode: int = SORT_SLICED, stats: bool = True) -> dict | None:
    """tigas_render_ex; returns the frame statistics (stats=False passes no
    statistics struct, so the uninstrumented kernels run, and returns None)."""
    fs = FrameStats() if stats else None
    _check(load_library().tigas_render_ex(scene.handle, ctypes.byref(make_pose(pose)),
                                          ctypes.byref(make_intrinsics(intr)), width, height, _ptr(out_rgba8),
                                          _ptr(out_rgba_f32), _stream(stream), sort_mode,
                                          ctypes.byref(fs) if stats else None))
    return _stats_dict(fs) if stats else None


def render_batch(scene: SceneHandle, poses: Sequence, intrs: Sequence, widths: Sequence[int],
                 heights: Sequence[int], outs: Sequence, stream=None, sort_mode: int | None = None):
    """tigas_render_batch: all views in one fused launch set.  With sort_mode
    given, tigas_render_batch_ex is called and its statistics returned."""
    V = len(poses)
    P = (Pose * V)(*[make_pose(p) for p in poses])
    K = (Intrinsics * V)(*[make_intrinsics(k) for k in intrs])
    W = (ctypes.c_int * V)(*widths)
    H = (ctypes.c_int * V)(*heights)
    O = (ctypes.c_void_p * V)(*[_ptr(o) for o in outs])
    if sort_mode is not None:
        stats = FrameStats()
        _check(load_library().tigas_render_batch_ex(scene.handle, V, P, K, ctypes.cast(W, ctypes.c_void_p),
                                                    ctypes.cast(H, ctypes.c_void_p), ctypes.cast(O, ctypes.c_void_p),
                                                    _stream(stream), sort_mode, ctypes.byref(stats)))
        return _stats_dict(stats)
    _check(load_library().tigas_render_batch(scene.handle, V, P, K, ctypes.cast(W, ctypes.c_void_p),
                                             ctypes.cast(H, ctypes.c_void_p), ctypes.cast(O, ctypes.c_void_p),
                                             _stream(stream)))
    return None


class RenderTicket:
    """An enqueued launch set (tigas_render_batch_async); wait() completes it."""

    def __init__(self, handle: int, keep):
        self.handle = handle
        self._keep = keep   # the output tensors stay referenced until the wait

    def wait(self) -> None:
        if self.handle:
            h, self.handle = self.handle, None
            self._keep = None
            _check(load_library().tigas_render_wait(h))


def render_batch_async(scene: SceneHandle, poses: Sequence, intrs: Sequence, widths: Sequence[int],
                       heights: Sequence[int], outs: Sequence, stream=None) -> RenderTicket:
    """tigas_render_batch_async: enqueue one launch set (device outputs, or
    pinned host outputs copied back on the ticket's copy stream)."""
    V = len(poses)
    P = (Pose * V)(*[make_pose(p) for p in poses])
    K = (Intrinsics * V)(*[make_intrinsics(k) for k in intrs])
    W = (ctypes.c_int * V)(*widths)
    H = (ctypes.c_int * V)(*heights)
    O = (ctypes.c_void_p * V)(*[_ptr(o) for o in outs])
    t = ctypes.c_void_p()
    _check(load_library().tigas_render_batch_async(scene.handle, V, P, K, ctypes.cast(W, ctypes.c_void_p),
                                                   ctypes.cast(H, ctypes.c_void_p), ctypes.cast(O, ctypes.c_void_p),
                                                   _stream(stream), ctypes.byref(t)))
    return RenderTicket(t.value, list(outs))


# The largest view count of each launch-set class with its own schedule (1, 2, 3-4, 5-8, ...).
SCHEDULE_CLASSES = (1, 2, 4, 8, 16, 32, 64)


def set_schedule(n_slices: int = 8, first_slice_inv: int = 64, blend_ctas_per_sm: int = 0, blend_batch: int = 32,
                 views_per_set: int = 0, n_views: int = 0) -> None:
    """tigas_set_schedule (n_views 0: every launch-set class) or
    tigas_set_schedule_for_views (the class of n_views only)."""
    s = Schedule(n_slices, first_slice_inv, blend_ctas_per_sm, blend_batch, views_per_set)
    lib = load_library()
    _check(lib.tigas_set_schedule(ctypes.byref(s)) if n_views == 0 else
           lib.tigas_set_schedule_for_views(n_views, ctypes.byref(s)))


def get_schedule(n_views: int = 1) -> dict:
    """tigas_get_schedule: the schedule of launch sets of n_views views."""
    s = Schedule()
    _check(load_library().tigas_get_schedule(n_views, ctypes.byref(s)))
    return s.as_dict()


def get_schedules() -> dict:
    """Every class's schedule, keyed by its largest view count (for set_schedules)."""
    return {n: get_schedule(n) for n in SCHEDULE_CLASSES}


def set_schedules(schedules: dict) -> None:
    """Sets each class's schedule from get_schedules()'s result."""
    for n, s in schedules.items():
        set_schedule(**s, n_views=n)


def jpeg_encode(rgba, quality: int, restart_mcus: int = 2, out=None, stream=None) -> bytes | int:
    """tigas_jpeg_encode of an [H, W, 4] uint8 frame (host array or device
    tensor).  Without ``out`` returns the file as bytes; with a caller buffer
    (host or device) returns the file length."""
    H, W = int(rgba.shape[0]), int(rgba.shape[1])
    n = ctypes.c_uint64()
    if out is None:
        buf = np.zeros(1024 + H * W * 4, np.uint8)
        _check(load_library().tigas_jpeg_encode(_ptr(rgba), W, H, quality, restart_mcus, _ptr(buf), buf.nbytes,
                                                ctypes.byref(n), _stream(stream)))
        return buf[:n.value].tobytes()
    cap = out.nbytes if hasattr(out, "nbytes") else out.numel() * out.element_size()
    _check(load_library().tigas_jpeg_encode(_ptr(rgba), W, H, quality, restart_mcus, _ptr(out), cap, ctypes.byref(n),
                                            _stream(stream)))
    return int(n.value)


def exact_rerenders() -> int:
    """Fixed-capacity launch sets that overflowed and were rendered again exactly."""
    return int(load_library().tigas_exact_rerenders())


def autotune(scene: SceneHandle, pose_sets: Sequence[Sequence], intrs: Sequence, widths: Sequence[int],
             heights: Sequence[int], outs: Sequence, iters: int = 3) -> tuple[dict, float]:
    """tigas_autotune: time the candidate schedules on launch sets of these
    resolutions, cycling through pose_sets (each a list of one pose per view),
    and keep the fastest; returns (schedule, median device ms per launch set)."""
    V = len(widths)
    S = len(pose_sets)
    if any(len(ps) != V for ps in pose_sets) or len(intrs) != V:
        raise ValueError("every pose set and the intrinsics need one entry per view")
    P = (Pose * (S * V))(*[make_pose(p) for ps in pose_sets for p in ps])
    K = (Intrinsics * (S * V))(*[make_intrinsics(k) for _ in range(S) for k in intrs])
    W = (ctypes.c_int * V)(*widths)
    H = (ctypes.c_int * V)(*heights)
    O = (ctypes.c_void_p * V)(*[_ptr(o) for o in outs])
    best = Schedule()
    ms = ctypes.c_double()
    _check(load_library().tigas_autotune(scene.handle, S, V, P, K, W, H, O, iters, ctypes.byref(best),
                                         ctypes.byref(ms)))
    return best.as_dict(), float(ms.value)


def debug_render(scene: SceneHandle, pose, intr, width: int, height: int, sort_mode: int = SORT_DEPTH_FIRST,
                 pair_capacity: int | None = None) -> dict:
    """tigas_debug_render: per-Gaussian decisions, sorted tile lists, ranges, float frame."""
    n = scene.n
    tx, ty = (width + 15) // 16, (height + 15) // 16
    cap = pair_capacity if pair_capacity is not None else max(1, 64 * n)
    out = {
        "visible": np.zeros(n, np.uint8), "radius": np.zeros(n, np.int32), "rect": np.zeros((n, 4), np.int32),
        "depth": np.zeros(n, np.float32), "uv": np.zeros((n, 2), np.float32), "q": np.zeros(n, np.float32),
        "values": np.zeros(cap, np.uint32), "ranges": np.zeros((tx * ty, 2), np.uint32),
        "rgba_f32": np.zeros((height, width, 4), np.float32),
    }
    lists = sort_mode != SORT_SLICED
    if not lists:
        out["values"] = np.zeros(0, np.uint32)
        out["ranges"] = np.zeros((0, 2), np.uint32)
    d = DebugFrame(*[_ptr(out[k]) for k in ["visible", "radius", "rect", "depth", "uv", "q"]],
                   _ptr(out["values"]) if lists else None, cap, _ptr(out["ranges"]) if lists else None,
                   _ptr(out["rgba_f32"]))
    pairs = ctypes.c_uint64()
    _check(load_library().tigas_debug_render(scene.handle, ctypes.byref(make_pose(pose)),
                                             ctypes.byref(make_intrinsics(intr)), width, height, sort_mode,
                                             ctypes.byref(d), ctypes.byref(pairs)))
    P = int(pairs.value)
    if lists and P > cap:
        return debug_render(scene, pose, intr, width, height, sort_mode, P)
    out["pairs"] = P
    if lists:
        out["values"] = out["values"][:P]
    return out


def sort_pairs_u64(keys_in, values_in, keys_out, values_out, n: int, begin_bit: int = 0, end_bit: int = 64,
                   stream=None) -> None:
    """tigas_sort_pairs_u64 on device buffers (torch tensors or raw pointers)."""
    _check(load_library().tigas_sort_pairs_u64(_ptr(keys_in), _ptr(values_in), _ptr(keys_out), _ptr(values_out),
                                               n, begin_bit, end_bit, _stream(stream)))


# ---------------------------------------------------------------- server


@dataclass
class ServerCompletion:
    ticket: int
    client_id: int
    status: int
    width: int
    height: int
    submit_us: float
    admit_us: float
    done_us: float


class Server:
    """tigas_server: continuous batching of per-client render requests."""

    def __init__(self, hbm_budget_bytes: int = 0, max_batch: int = 0, max_inflight: int = 0,
                 batch_window_us: int = 0):
        cfg = ServerConfig(hbm_budget_bytes, max_batch, max_inflight, batch_window_us)
        h = ctypes.c_void_p()
        _check(load_library().tigas_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self.handle = h.value
        self._keep: dict[int, Any] = {}

    def submit(self, scene: SceneHandle, pose, intr, width: int, height: int, out, client_id: int) -> int:
        t = ctypes.c_uint64()
        _check(_lib.tigas_server_submit(self.handle, scene.handle, ctypes.byref(make_pose(pose)),
                                        ctypes.byref(make_intrinsics(intr)), width, height, _ptr(out), client_id,
                                        ctypes.byref(t)))
        self._keep[t.value] = out
        return int(t.value)

    def poll(self, max_n: int = 256, timeout_us: int = 0) -> list[ServerCompletion]:
        buf = (Completion * max_n)()
        k = ctypes.c_int()
        _check(_lib.tigas_server_poll(self.handle, buf, max_n, timeout_us, ctypes.byref(k)))
        res = []
        for c in buf[:k.value]:
            self._keep.pop(c.ticket, None)
            res.append(ServerCompletion(c.ticket, c.client_id, c.status, c.width, c.height, c.submit_us,
                                        c.admit_us, c.done_us))
        return res

    def destroy(self, cancel: bool = False) -> None:
        if self.handle:
            _check(_lib.tigas_server_destroy(self.handle, int(cancel)))
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()
