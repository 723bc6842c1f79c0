"""CPU oracle of the frame encoder (baseline JPEG in a JFIF file) that
follows the blend: the response payload of a render request (Sec. 4.1, 5.1;
the quality levels of Table 1).  Test infrastructure: only the tests,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU leg use it; it shares no
code with the CUDA encoder.  ``jpeg.c`` states the encoding step by step.

Parity status: pinned by ``tests/test_oracle_jpeg.py`` (the fixed-point DCT
against the double-precision FDCT definition, the quantizer tables against
their definition, and the bitstream through an independent decoder:
constant images decode to their exact colour, smooth images round-trip
within the quantization error, restart intervals and byte stuffing parse).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "jpeg.c")
_LIB = os.path.join(_HERE, "_jpeg.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=gnu11", "-ffp-contract=off", _SRC, "-o", tmp,
                               "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            lib.oracle_jpeg_encode.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P,
                                               ctypes.c_int64]
            lib.oracle_jpeg_encode.restype = ctypes.c_int64
            lib.oracle_jpeg_quant_table.argtypes = [ctypes.c_int, ctypes.c_int, P]
            lib.oracle_jpeg_fdct_fixed.argtypes = [P, P]
            lib.oracle_jpeg_fdct_exact.argtypes = [P, P]
            _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def encode(rgba: np.ndarray, quality: int, restart: int = 4) -> bytes:
    """JPEG file of an [H, W, 4] uint8 image (alpha ignored); restart: MCUs per interval."""
    img = np.ascontiguousarray(rgba, dtype=np.uint8)
    H, W = img.shape[:2]
    lib = _load()
    cap = 1024 + H * W * 8
    out = np.zeros(cap, np.uint8)
    n = lib.oracle_jpeg_encode(_p(img), W, H, int(quality), int(restart), _p(out), cap)
    if n < 0 or n > cap:
        raise ValueError("bad image size or output capacity")
    return out[:n].tobytes()


def quant_table(quality: int, chroma: bool) -> np.ndarray:
    q = np.zeros(64, np.int32)
    _load().oracle_jpeg_quant_table(int(quality), int(chroma), _p(q))
    return q.reshape(8, 8)


def fdct_fixed(block: np.ndarray) -> np.ndarray:
    """Level-shifted 8x8 block -> coefficients x 2^16 (fixed-point path)."""
    s = np.ascontiguousarray(block, dtype=np.int32).reshape(64)
    out = np.zeros(64, np.int32)
    _load().oracle_jpeg_fdct_fixed(_p(s), _p(out))
    return out.reshape(8, 8)


def fdct_exact(block: np.ndarray) -> np.ndarray:
    s = np.ascontiguousarray(block, dtype=np.int32).reshape(64)
    out = np.zeros(64, np.float64)
    _load().oracle_jpeg_fdct_exact(_p(s), _p(out))
    return out.reshape(8, 8)
