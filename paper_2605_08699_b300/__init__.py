"""B300-native forward 3D Gaussian Splatting renderer behind a C ABI.

The compute path lives in ``libtigas.so`` (``csrc/``, sm_103a CUDA); this
package is its Python binding (``tigas.py``) and build script (``build.py``).
"""
from .tigas import (SORT_DEPTH_FIRST, SORT_FULL64, SORT_SLICED, STORAGE_FP16, STORAGE_FP32, TigasError, Server, SceneHandle,
                    debug_render, kernel_launches, last_error, load_library, make_intrinsics, profile_enable, profile_read, set_graphs, make_pose, render,
                    render_batch, render_ex, scene_from, scene_load, sort_pairs_u64, version)

__all__ = ["SORT_DEPTH_FIRST", "SORT_FULL64", "SORT_SLICED", "STORAGE_FP16", "STORAGE_FP32", "TigasError", "Server", "SceneHandle",
           "debug_render", "kernel_launches", "last_error", "load_library", "make_intrinsics", "profile_enable", "profile_read", "set_graphs", "make_pose", "render",
           "render_batch", "render_ex", "scene_from", "scene_load", "sort_pairs_u64", "version"]
