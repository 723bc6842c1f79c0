"""B300-native forward 3D Gaussian Splatting renderer behind a C ABI.

The compute path lives in ``libtigas.so`` (``csrc/``, sm_103a CUDA); this
package is its Python binding (``tigas.py``), the serving loop's resolution
controller (``abr.py``) and the build script (``build.py``).
"""
from .tigas import (ERR_AGAIN, ERR_CUDA, ERR_INVALID, ERR_IO, ERR_NOT_FOUND, ERR_OOM, ERR_OVERFLOW, ERR_TIMEOUT, OK,
                    SORT_DEPTH_FIRST, SORT_FULL64, SORT_SLICED, STAGES, STORAGE_FP16, STORAGE_FP32, Registry,
                    RegistryScene, SceneHandle, Server, TigasError, autotune, debug_render, debug_sort_wait_timeout, exact_rerenders, get_schedule, jpeg_encode,
                    kernel_launches, last_error, load_library, make_intrinsics, make_pose, profile_enable,
                    image_quality, ply_decode, ply_probe, profile_read, profile_stages, render, render_batch, render_batch_async, RenderTicket, render_ex, scene_from, scene_load,
                    scene_load_ply, set_graphs, set_schedule, sort_pairs_u64, resample_rgba8, version,
                    DEVICE_ALLOC, PINNED_ALLOC, debug_fail_alloc, release_workspace, SCHEDULE_CLASSES,
                    get_schedules, set_schedules)

__all__ = ["ERR_AGAIN", "ERR_CUDA", "ERR_INVALID", "ERR_IO", "ERR_NOT_FOUND", "ERR_OOM", "ERR_OVERFLOW", "ERR_TIMEOUT", "OK",
           "SORT_DEPTH_FIRST", "SORT_FULL64", "SORT_SLICED", "STAGES", "STORAGE_FP16", "STORAGE_FP32", "Registry",
           "RegistryScene", "SceneHandle",
           "Server", "TigasError", "autotune", "debug_render", "debug_sort_wait_timeout", "exact_rerenders", "get_schedule", "jpeg_encode",
           "kernel_launches", "last_error", "load_library", "make_intrinsics", "make_pose", "profile_enable",
           "image_quality", "ply_decode", "ply_probe", "profile_read", "profile_stages", "render", "render_batch", "render_batch_async", "RenderTicket", "render_ex", "scene_from", "scene_load",
           "scene_load_ply", "set_graphs",
           "set_schedule", "sort_pairs_u64", "resample_rgba8", "version",
           "DEVICE_ALLOC", "PINNED_ALLOC", "debug_fail_alloc", "release_workspace", "SCHEDULE_CLASSES", "get_schedules", "set_schedules"]
