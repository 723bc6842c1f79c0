"""PLY reading and model-registry scanning on the CPU.

The reference reader (oracle/ply.py) is pinned by a hand-written ASCII file
whose expected arrays are spelled out below, and by round trips of the
synthetic writer across formats, property types, orders and extra elements.
The library's header parser (tigas_ply_probe) and the registry's folder scan
need no GPU and are checked here; decoding and loading are GPU tests."""
import ctypes
import os

import numpy as np
import pytest

import paper_2605_08699_b300 as tg
import synth
from oracle import ply as oply
from synth import ply as sply

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "ply_tiny_ascii.ply")


def _scene(n=37, degree=3, seed=7):
    return synth.make_scene(n, synth.BASE_SEED + seed, n_blobs=4, sh_degree=degree)


def test_golden_ascii_file():
    """Two Gaussians of degree 1 written by hand with the properties out of
    order: rot_0 is the real part, f_rest is channel-major (M = 3)."""
    r = oply.read_ply(GOLDEN)
    assert r["sh_degree"] == 1
    np.testing.assert_array_equal(r["means"], np.float32([[0.5, -1.25, 2], [-0.5, 1.25, -2]]))
    np.testing.assert_array_equal(r["log_scales"], np.float32([[-3, -4, -5], [0.25, 0.5, 0.75]]))
    np.testing.assert_array_equal(r["quats"], np.float32([[1, 0, 0, 0], [0.5, 0.5, -0.5, 0.5]]))
    np.testing.assert_array_equal(r["opacity_logits"], np.float32([-2, 3]))
    sh = np.zeros((2, 16, 3), np.float32)
    sh[0, 0] = np.float32([0.1, 0.2, 0.3])
    sh[1, 0] = np.float32([1.1, 1.2, 1.3])
    for v, base in ((0, 100), (1, 200)):
        for c in range(3):
            for j in range(3):
                sh[v, 1 + j, c] = base + 3 * c + j
    np.testing.assert_array_equal(r["sh"], sh)


def test_probe_golden_file():
    info = tg.ply_probe(GOLDEN)
    assert info["n"] == 2 and info["sh_degree"] == 1 and info["format"] == "ascii"
    assert info["n_properties"] == 24


VARIANTS = [
    dict(fmt="binary_little_endian"),
    dict(fmt="binary_big_endian"),
    dict(fmt="ascii"),
    dict(fmt="binary_little_endian", shuffle_seed=3, extra_elements=True),
    dict(fmt="binary_big_endian", shuffle_seed=4, extra_elements=True, normals=False),
    dict(fmt="ascii", shuffle_seed=5, extra_elements=True),
    dict(fmt="binary_little_endian", types={"x": "double", "opacity": "double", "f_rest_7": "double",
                                            "nx": "uchar"}),
]


@pytest.mark.parametrize("degree", [0, 1, 2, 3])
@pytest.mark.parametrize("k", range(len(VARIANTS)))
def test_writer_reader_round_trip(tmp_path, k, degree):
    sc = _scene(degree=degree, seed=10 + k)
    path = tmp_path / "s.ply"
    sply.write_ply(path, sc, **VARIANTS[k])
    r = oply.read_ply(path)
    assert r["sh_degree"] == degree
    for name in ("means", "log_scales", "quats", "opacity_logits"):
        np.testing.assert_array_equal(r[name], getattr(sc, name))
    want = sc.sh.copy()
    want[:, (degree + 1) ** 2:, :] = 0
    np.testing.assert_array_equal(r["sh"], want)
    info = tg.ply_probe(path)
    assert info["n"] == sc.n and info["sh_degree"] == degree and info["format"] == VARIANTS[k]["fmt"]
    n_props = len(sply.vertex_columns(sc, degree, VARIANTS[k].get("normals", True)))
    assert info["n_properties"] == n_props
    if VARIANTS[k]["fmt"] != "ascii":
        sizes = {"double": 8, "uchar": 1}
        types = VARIANTS[k].get("types", {})
        row = sum(sizes.get(types.get(name, "float"), 4)
                  for name, _ in sply.vertex_columns(sc, degree, VARIANTS[k].get("normals", True)))
        assert info["row_bytes"] == row
        extra = 2 * 5 if VARIANTS[k].get("extra_elements") else 0
        assert info["file_bytes"] - info["body_offset"] - sc.n * row == (13 if extra else 0)


def test_integer_property_types_round(tmp_path):
    sc = _scene(n=9, degree=0)
    sc.opacity_logits[:] = np.float32([-3.4, -2.6, -1.5, 0.49, 0.5, 1.5, 2.5, 7.2, 100.7])
    path = tmp_path / "i.ply"
    sply.write_ply(path, sc, types={"opacity": "short"})
    r = oply.read_ply(path)
    np.testing.assert_array_equal(r["opacity_logits"], np.rint(sc.opacity_logits))


def _write_header(path, lines, body=b""):
    with open(path, "wb") as f:
        f.write(("\n".join(lines) + "\n").encode() + body)


_PROPS = ["x", "y", "z", "f_dc_0", "f_dc_1", "f_dc_2", "opacity", "scale_0", "scale_1", "scale_2",
          "rot_0", "rot_1", "rot_2", "rot_3"]


def _header(props, n=1, fmt="binary_little_endian", pre=(), post=()):
    return ["ply", f"format {fmt} 1.0", *pre, f"element vertex {n}"] + [f"property float {p}" for p in props] + \
        list(post) + ["end_header"]


def _probe_status(path):
    info = tg.tigas.PlyInfo()
    return tg.load_library().tigas_ply_probe(os.fsencode(str(path)), ctypes.byref(info)), info


def test_probe_accepts_minimal_degree0(tmp_path):
    p = tmp_path / "ok.ply"
    _write_header(p, _header(_PROPS, n=2), bytes(2 * 4 * len(_PROPS)))
    st, info = _probe_status(p)
    assert st == tg.OK and info.n == 2 and info.sh_degree == 0 and info.row_bytes == 56


@pytest.mark.parametrize("case", ["missing_rot3", "rest10", "rest_gap", "truncated", "vertex_list", "pre_list",
                                  "not_ply", "no_end", "bad_type", "zero_n", "dup", "bad_format"])
def test_probe_rejects_bad_headers(tmp_path, case):
    p = tmp_path / f"{case}.ply"
    props = list(_PROPS)
    lines = None
    body = bytes(4 * len(props))
    if case == "missing_rot3":
        props.remove("rot_3")
    elif case == "rest10":
        props += [f"f_rest_{k}" for k in range(10)]
    elif case == "rest_gap":
        props += [f"f_rest_{k}" for k in range(9) if k != 4] + ["f_rest_9"]
    elif case == "dup":
        props += ["x"]
    if case == "truncated":
        body = bytes(4 * len(props) - 1)
    body = bytes(4 * len(props)) if case not in ("truncated",) else body
    lines = _header(props)
    if case == "vertex_list":
        lines = _header(props, post=["property list uchar int idx"])
    elif case == "pre_list":
        lines = _header(props, pre=["element face 1", "property list uchar int vertex_indices"])
    elif case == "not_ply":
        lines = ["plx"] + lines[1:]
    elif case == "no_end":
        lines = lines[:-1]
    elif case == "bad_type":
        lines = [ln.replace("property float y", "property float16 y") for ln in lines]
    elif case == "zero_n":
        lines = _header(props, n=0)
    elif case == "bad_format":
        lines = _header(props, fmt="binary_middle_endian")
    _write_header(p, lines, body)
    st, _ = _probe_status(p)
    assert st == tg.ERR_INVALID, (case, tg.last_error())


def test_probe_missing_file_is_io_error(tmp_path):
    st, _ = _probe_status(tmp_path / "absent.ply")
    assert st == tg.ERR_IO


def test_ascii_list_element_before_vertex_is_skipped(tmp_path):
    p = tmp_path / "a.ply"
    sc = _scene(n=3, degree=0)
    sply.write_ply(p, sc, fmt="ascii", extra_elements=True)
    assert tg.ply_probe(p)["n"] == 3


# ------------------------------------------------------------------ registry


def _model_tree(root):
    """a/ (two training iterations + preview), b/ (a loose PLY), c.ply + c.png,
    d.ply beside folder d/ (the folder wins), broken.ply, empty/ (no PLY)."""
    sizes = {}
    for it, n in ((7000, 11), (30000, 13)):
        d = root / "a" / "point_cloud" / f"iteration_{it}"
        d.mkdir(parents=True)
        sply.write_ply(d / "point_cloud.ply", _scene(n=n, degree=3))
    (root / "a" / "preview.jpg").write_bytes(b"\xff\xd8\xff\xd9")
    (root / "b").mkdir()
    sply.write_ply(root / "b" / "scene.ply", _scene(n=17, degree=1))
    sply.write_ply(root / "c.ply", _scene(n=19, degree=0))
    (root / "c.png").write_bytes(b"\x89PNG")
    (root / "d").mkdir()
    sply.write_ply(root / "d" / "m.ply", _scene(n=23, degree=2))
    sply.write_ply(root / "d.ply", _scene(n=29, degree=2))
    (root / "broken.ply").write_bytes(b"ply\nformat ascii 1.0\nend_header\n")
    (root / "empty").mkdir()
    return sizes


def test_registry_scan_metadata(tmp_path):
    _model_tree(tmp_path)
    with tg.Registry(tmp_path, idle_timeout_s=5.0) as reg:
        ms = reg.models()
        assert [m["id"] for m in ms] == ["a", "b", "c", "d"]
        a, b, c, d = ms
        assert a["ply_path"].endswith(os.path.join("iteration_30000", "point_cloud.ply")) and a["n"] == 13
        assert a["preview_path"].endswith(os.path.join("a", "preview.jpg")) and a["sh_degree"] == 3
        assert b["ply_path"].endswith(os.path.join("b", "scene.ply")) and b["n"] == 17 and b["preview_path"] == ""
        assert c["ply_path"].endswith("c.ply") and c["preview_path"].endswith("c.png") and c["sh_degree"] == 0
        assert d["ply_path"].endswith(os.path.join("d", "m.ply")) and d["n"] == 23
        for m in ms:
            assert not m["loaded"] and m["users"] == 0 and m["loads"] == 0 and m["resident_bytes"] == 0
            assert m["name"] == m["id"] and m["file_bytes"] == os.path.getsize(m["ply_path"])
        sply.write_ply(tmp_path / "e.ply", _scene(n=5, degree=0))
        assert reg.scan() == (5, 1)   # broken.ply is skipped
        assert reg.models()[-1]["id"] == "e"
        os.remove(tmp_path / "c.ply")
        assert reg.scan() == (4, 1)
        assert [m["id"] for m in reg.models()] == ["a", "b", "d", "e"]


def test_registry_errors_without_gpu(tmp_path):
    with pytest.raises(tg.TigasError) as e:
        tg.Registry(tmp_path / "nope")
    assert e.value.status == tg.ERR_IO
    with pytest.raises(tg.TigasError) as e:
        tg.Registry(tmp_path, idle_timeout_s=-1)
    assert e.value.status == tg.ERR_INVALID
    with tg.Registry(tmp_path) as reg:
        assert len(reg) == 0
        with pytest.raises(tg.TigasError) as e:
            reg.acquire("missing")
        assert e.value.status == tg.ERR_NOT_FOUND
        with pytest.raises(tg.TigasError):
            reg.info(0)
        assert reg.evict_idle() == 0
        with pytest.raises(tg.TigasError):
            reg.start_eviction(0.0)
