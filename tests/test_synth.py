"""Seeded input generators: Philox known answers, determinism, distributions."""
import math
import os

import numpy as np

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_philox_known_answers():
    for row in _read_rows("philox4x32_10_kat.txt"):
        w = [int(x, 16) for x in row]
        assert synth.philox4x32_10(w[0:4], w[4:6]) == tuple(w[6:10])


def test_scene_deterministic_and_chunk_free():
    a = synth.make_scene(5000, 123, n_blobs=8, iso_sigma=0.3)
    b = synth.make_scene(5000, 123, n_blobs=8, iso_sigma=0.3)
    c = synth.make_scene(7000, 123, n_blobs=8, iso_sigma=0.3)   # prefix must match
    for x, y, z in [(a.means, b.means, c.means), (a.sh, b.sh, c.sh), (a.quats, b.quats, c.quats)]:
        assert np.array_equal(x, y)
        assert np.array_equal(x, z[:5000])
    d = synth.make_scene(5000, 124, n_blobs=8, iso_sigma=0.3)
    assert not np.array_equal(a.means, d.means)


def test_scene_distributions():
    s = synth.make_scene(200_000, 7, n_blobs=64)
    assert np.all(np.abs(s.means) <= 1.0)
    assert abs(s.log_scales.mean() + 4.0) < 0.01 and abs(s.log_scales.std() - 0.5) < 0.01
    assert abs(s.opacity_logits.mean()) < 0.02 and abs(s.opacity_logits.std() - 1.5) < 0.02
    assert abs(s.sh[:, 0, :].std() - 0.5) < 0.01 and abs(s.sh[:, 1:, :].std() - 0.05) < 0.001
    assert abs(s.quats.std() - 1.0) < 0.01
    # isotropic blobs of sigma 0.3 (before the cube rejection trims the tails)
    t = synth.make_scene(100_000, 9, n_blobs=1, iso_sigma=0.3)
    centred = t.means - np.median(t.means, axis=0)
    assert 0.25 < centred.std() < 0.31


def test_normals_moments():
    z = synth.normals(1, 2, 400_000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01
    u = synth.uniforms(1, 3, 400_000)
    assert u.min() > 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01


def test_trajectory_random_walk():
    tr = synth.trajectory(99, 300)
    assert len(tr) == 300
    assert tr[0].t == synth.BASE_POSE.t and tr[0].azimuth == 0.0
    steps = np.diff(np.array([p.t for p in tr]), axis=0)
    assert abs(steps.std() - 0.01) < 0.002
    az = np.diff([p.azimuth for p in tr])
    assert abs(np.degrees(az).std() - 0.5) < 0.1
    assert all(abs(p.elevation) <= math.radians(80) + 1e-12 for p in tr)


def test_default_camera_and_ladders():
    k = synth.default_intrinsics(1920, 1080)
    assert abs(k.fy - 1080 / (2 * math.tan(math.radians(30)))) < 1e-9
    assert (k.cx, k.cy) == (960.0, 540.0)
    # f x 1920x1080 for f in {0.25, 0.4, 0.5, 2/3, 0.8, 1}
    for (w, h), f in zip(synth.ABR_LEVELS, [0.25, 0.4, 0.5, 2 / 3, 0.8, 1.0]):
        assert (w, h) == (round(1920 * f), round(1080 * f))
    rows = [tuple(int(x) for x in r) for r in _read_rows("table1_bitrate_ladder.txt")]
    assert rows == synth.TABLE1_LADDER
