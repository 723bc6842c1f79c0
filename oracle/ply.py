"""Reference PLY reader for 3DGS scenes (test infrastructure).

Only the tests and bench.py's CPU legs use it.  It reads a PLY file with
plain numpy -- a structured dtype over the binary vertex block, or a float
parse of each ASCII token -- and returns the raw per-Gaussian attributes of
Sec. 5.1 ("PLY Model and Primitives"): means [N,3], log-scales [N,3],
quaternions [N,4] (w, x, y, z = rot_0..3), opacity logits [N] and SH
coefficients [N,16,3].  The SH layout follows the file convention of the
3DGS reference implementation that Sec. 4.1 builds on: f_dc_c is coefficient
0 of channel c and f_rest_{c*M+j} is coefficient j+1 of channel c, with
M = (d+1)^2 - 1 and the degree d given by the f_rest count.  Values become
float32 by round-to-nearest.

Parity pins: tests/golden/ply_tiny_ascii.ply (hand-written, with its
expected arrays in the test) and round trips of synth.ply's writer across
formats, property types and orders.
"""
from __future__ import annotations

import numpy as np

_TYPES = {"char": "i1", "int8": "i1", "uchar": "u1", "uint8": "u1", "short": "i2", "int16": "i2",
          "ushort": "u2", "uint16": "u2", "int": "i4", "int32": "i4", "uint": "u4", "uint32": "u4",
          "float": "f4", "float32": "f4", "double": "f8", "float64": "f8"}


def _header(data: bytes):
    end = data.index(b"end_header\n") + len(b"end_header\n")
    lines = data[:end].decode("ascii").splitlines()
    assert lines[0] == "ply"
    fmt, elems = None, []
    for line in lines[1:-1]:
        tok = line.split()
        if not tok or tok[0] in ("comment", "obj_info"):
            continue
        if tok[0] == "format":
            fmt = tok[1]
        elif tok[0] == "element":
            elems.append({"name": tok[1], "count": int(tok[2]), "props": []})
        elif tok[0] == "property":
            if tok[1] == "list":
                elems[-1]["props"].append(("list", tok[4]))
            else:
                elems[-1]["props"].append((_TYPES[tok[1]], tok[2]))
    return fmt, elems, end


def read_ply(path) -> dict:
    """Raw attributes of a 3DGS PLY: dict with means, log_scales, quats,
    opacity_logits, sh (float32) and sh_degree."""
    with open(path, "rb") as f:
        data = f.read()
    fmt, elems, pos = _header(data)
    cols = {}
    if fmt == "ascii":
        rows = data[pos:].decode("ascii").splitlines()
        k = 0
        for e in elems:
            if e["name"] == "vertex":
                names = [p[1] for p in e["props"]]
                vals = np.array([[float(t) for t in rows[k + i].split()] for i in range(e["count"])], np.float64)
                cols = {name: vals[:, j] for j, name in enumerate(names)}
                break
            k += e["count"]
    else:
        end = "<" if fmt == "binary_little_endian" else ">"
        for e in elems:
            if e["name"] == "vertex":
                dt = np.dtype([(name, end + t) for t, name in e["props"]])
                rec = np.frombuffer(data, dtype=dt, count=e["count"], offset=pos)
                cols = {name: rec[name] for _, name in e["props"]}
                break
            assert all(t != "list" for t, _ in e["props"])
            pos += e["count"] * np.dtype([(name, end + t) for t, name in e["props"]]).itemsize
    f32 = lambda name: np.asarray(cols[name]).astype(np.float32)
    n = len(cols["x"])
    n_rest = sum(1 for name in cols if name.startswith("f_rest_"))
    degree = {0: 0, 9: 1, 24: 2, 45: 3}[n_rest]
    M = (degree + 1) ** 2 - 1
    sh = np.zeros((n, 16, 3), np.float32)
    for c in range(3):
        sh[:, 0, c] = f32(f"f_dc_{c}")
        for j in range(M):
            sh[:, 1 + j, c] = f32(f"f_rest_{c * M + j}")
    return {"means": np.stack([f32("x"), f32("y"), f32("z")], 1),
            "log_scales": np.stack([f32(f"scale_{k}") for k in range(3)], 1),
            "quats": np.stack([f32(f"rot_{k}") for k in range(4)], 1),
            "opacity_logits": f32("opacity"), "sh": sh, "sh_degree": degree}
