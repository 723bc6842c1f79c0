"""Write synthetic scenes as 3DGS PLY files (test and benchmark inputs).

The files follow the vertex layout that 3DGS training writes: x y z, nx ny nz,
f_dc_0..2, f_rest_0..(3M-1) (channel-major: f_rest_{c*M+j} is SH coefficient
j + 1 of colour channel c, M = (d+1)^2 - 1), opacity, scale_0..2, rot_0..3.
Options vary what a reader must cope with: the three PLY formats, property
types other than float, a shuffled property order, and extra elements before
and after the vertex element.  This module holds no rendering arithmetic.
"""
from __future__ import annotations

import numpy as np

from . import Scene, uniforms

_NP = {"char": "i1", "uchar": "u1", "short": "i2", "ushort": "u2", "int": "i4", "uint": "u4",
       "float": "f4", "double": "f8"}


def vertex_columns(scene: Scene, sh_degree: int | None = None, normals: bool = True) -> list[tuple[str, np.ndarray]]:
    """(property name, float32 column) pairs in the 3DGS order."""
    d = scene.sh_degree if sh_degree is None else sh_degree
    M = (d + 1) ** 2 - 1
    cols = [("x", scene.means[:, 0]), ("y", scene.means[:, 1]), ("z", scene.means[:, 2])]
    if normals:
        z = np.zeros(scene.n, np.float32)
        cols += [("nx", z), ("ny", z), ("nz", z)]
    cols += [(f"f_dc_{c}", scene.sh[:, 0, c]) for c in range(3)]
    cols += [(f"f_rest_{c * M + j}", scene.sh[:, 1 + j, c]) for c in range(3) for j in range(M)]
    cols += [("opacity", scene.opacity_logits)]
    cols += [(f"scale_{k}", scene.log_scales[:, k]) for k in range(3)]
    cols += [(f"rot_{k}", scene.quats[:, k]) for k in range(4)]
    return cols


def write_ply(path, scene: Scene, fmt: str = "binary_little_endian", sh_degree: int | None = None,
              types: dict | None = None, shuffle_seed: int | None = None, normals: bool = True,
              extra_elements: bool = False) -> None:
    """Write ``scene`` to ``path``.  types: property name -> PLY type (default
    float); integer types take the rounded value.  shuffle_seed: permute the
    property order.  extra_elements: add a 'camera' element (two scalar
    properties, 2 instances) before the vertex element and a 'face' element
    with a list property after it."""
    cols = vertex_columns(scene, sh_degree, normals)
    if shuffle_seed is not None:
        order = np.argsort(uniforms(shuffle_seed, 21, len(cols)), kind="stable")
        cols = [cols[k] for k in order]
    types = types or {}
    tnames = [types.get(name, "float") for name, _ in cols]
    n = scene.n
    head = ["ply", f"format {fmt} 1.0", "comment synthetic 3DGS scene"]
    if extra_elements:
        head += ["element camera 2", "property float focal", "property uchar id"]
    head.append(f"element vertex {n}")
    head += [f"property {t} {name}" for (name, _), t in zip(cols, tnames)]
    if extra_elements:
        head += ["element face 1", "property list uchar int vertex_indices"]
    head.append("end_header")
    with open(path, "wb") as f:
        f.write(("\n".join(head) + "\n").encode())
        if fmt == "ascii":
            if extra_elements:
                f.write(b"1.5 7\n2.5 9\n")
            lines = []
            for i in range(n):
                vals = []
                for (_, col), t in zip(cols, tnames):
                    v = col[i]
                    vals.append("%d" % int(np.rint(v)) if _NP[t][0] in "iu" else "%.17g" % float(v))
                lines.append(" ".join(vals))
            f.write(("\n".join(lines) + "\n").encode())
            if extra_elements:
                f.write(b"3 0 1 2\n")
            return
        end = "<" if fmt == "binary_little_endian" else ">"
        if extra_elements:
            cam = np.zeros(2, dtype=[("focal", end + "f4"), ("id", "u1")])
            cam["focal"] = [1.5, 2.5]
            cam["id"] = [7, 9]
            f.write(cam.tobytes())
        dt = np.dtype([(name, end + _NP[t]) for (name, _), t in zip(cols, tnames)])
        rec = np.zeros(n, dtype=dt)
        for (name, col), t in zip(cols, tnames):
            rec[name] = np.rint(col) if _NP[t][0] in "iu" else col
        f.write(rec.tobytes())
        if extra_elements:
            f.write(bytes([3]) + np.array([0, 1, 2], end + "i4").tobytes())
