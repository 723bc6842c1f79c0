"""Quality kernels and deterministic replay on the GPU.

The resampler is integer arithmetic and must match the oracle bit for bit;
SSIM is FP32 against the FP64 oracle (1e-3 per window position, 1e-5 on the
mean, from the rounding of 11-tap FP32 sums of centred samples below 2^14);
PSNR uses an exact squared-error sum.  Replay must reproduce the same bytes,
its JPEGs must be the oracle encoder's files of the same renders, and its
metrics must agree with the oracle's."""
import math
import zlib

import numpy as np
import pytest

import synth
from oracle import jpeg as ojpeg
from oracle import quality as oq

torch = pytest.importorskip("torch")
import paper_2605_08699_b300 as tg  # noqa: E402
from paper_2605_08699_b300 import replay as rp  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    tg.load_library()
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def scene(cuda):
    with tg.scene_from(synth.config_scene(2, n=200_000), storage=tg.STORAGE_FP16) as h:
        yield h


def _noise(h, w, seed):
    return np.random.default_rng(seed).integers(0, 256, (h, w, 4), dtype=np.uint8)


@pytest.mark.parametrize("src,dst", [((480, 270), (1920, 1080)), ((97, 61), (333, 197)), ((333, 197), (97, 61)),
                                     ((1, 1), (5, 3)), ((64, 48), (64, 48)), ((8192, 2), (16, 7)),
                                     ((3, 2), (8192, 4))])
def test_resample_matches_oracle_bit_exact(cuda, src, dst):
    w, h = src
    img = _noise(h, w, w * 7 + h)
    want = oq.resample(img, *dst)
    assert np.array_equal(tg.resample_rgba8(img, *dst), want)
    d_out = torch.empty((dst[1], dst[0], 4), dtype=torch.uint8, device=cuda)
    tg.resample_rgba8(torch.from_numpy(img).to(cuda), *dst, out=d_out)
    assert np.array_equal(d_out.cpu().numpy(), want)


def _check_quality(a, b, cuda):
    m = np.full((a.shape[0] - 10, a.shape[1] - 10), np.nan, np.float32)
    got = tg.image_quality(a, b, ssim_map=m)
    ref_map = oq.ssim_map(a, b).mean(axis=0)
    assert np.abs(m - ref_map).max() <= 1e-3
    assert abs(got["ssim"] - oq.ssim(a, b)) <= 1e-5
    want_psnr = oq.psnr(a, b)
    assert (got["psnr"] == want_psnr) if math.isinf(want_psnr) else abs(got["psnr"] - want_psnr) < 1e-9
    # device frames and map give the same numbers, bit for bit
    da, db = torch.from_numpy(a).to(cuda), torch.from_numpy(b).to(cuda)
    dm = torch.empty(m.shape, dtype=torch.float32, device=cuda)
    got2 = tg.image_quality(da, db, ssim_map=dm)
    assert got2 == got and np.array_equal(dm.cpu().numpy(), m)
    return got


@pytest.mark.parametrize("size", [(11, 11), (43, 19), (97, 61), (1920, 1080)])
def test_quality_of_rendered_frames(cuda, scene, size):
    w, h = size
    K = synth.default_intrinsics(w, h)
    pose = synth.config_trajectory(2)[5]
    gt = tg.render(scene, pose, K, w, h)
    lw, lh = max(1, w // 3), max(1, h // 3)
    low = tg.render(scene, pose, synth.default_intrinsics(lw, lh), lw, lh)
    up = oq.resample(low, w, h)
    got = _check_quality(gt, up, cuda)
    assert 0.0 < got["ssim"] < 1.0


def test_quality_noise_identity_and_constants(cuda):
    a, b = _noise(70, 90, 1), _noise(70, 90, 2)
    _check_quality(a, b, cuda)
    got = _check_quality(a, a, cuda)
    assert abs(got["ssim"] - 1.0) < 1e-6 and got["psnr"] == math.inf
    c0 = np.zeros((30, 40, 4), np.uint8)
    c1 = np.full((30, 40, 4), 255, np.uint8)
    got = _check_quality(c0, c1, cuda)
    assert abs(got["ssim"] - oq.C1 / (255 ** 2 + oq.C1)) < 1e-7


def test_quality_is_deterministic(cuda, scene):
    gt = tg.render(scene, synth.BASE_POSE, synth.default_intrinsics(640, 360), 640, 360)
    up = tg.resample_rgba8(tg.render(scene, synth.BASE_POSE, synth.default_intrinsics(320, 180), 320, 180), 640, 360)
    r = [tg.image_quality(gt, up) for _ in range(3)]
    assert r[0] == r[1] == r[2]


def test_quality_rejects_bad_sizes(cuda):
    a = np.zeros((10, 40, 4), np.uint8)
    with pytest.raises(tg.TigasError) as e:
        tg.image_quality(a, a)
    assert e.value.status == tg.ERR_INVALID
    with pytest.raises(tg.TigasError):
        tg.resample_rgba8(np.zeros((4, 4, 4), np.uint8), 0, 3)


def _png_pixels(data: bytes) -> np.ndarray:
    assert data[:8] == b"\x89PNG\r\n\x1a\n"
    pos, idat, w, h = 8, b"", 0, 0
    while pos < len(data):
        n = int.from_bytes(data[pos:pos + 4], "big")
        tag, body = data[pos + 4:pos + 8], data[pos + 8:pos + 8 + n]
        assert int.from_bytes(data[pos + 8 + n:pos + 12 + n], "big") == zlib.crc32(tag + body) & 0xFFFFFFFF
        if tag == b"IHDR":
            w, h = int.from_bytes(body[:4], "big"), int.from_bytes(body[4:8], "big")
            assert body[8:] == bytes([8, 6, 0, 0, 0])
        elif tag == b"IDAT":
            idat += body
        pos += 12 + n
    raw = np.frombuffer(zlib.decompress(idat), np.uint8).reshape(h, 1 + 4 * w)
    assert (raw[:, 0] == 0).all()
    return raw[:, 1:].reshape(h, w, 4)


def test_replay_materializes_deterministic_frames(cuda, scene, tmp_path):
    log = synth.pose_log(n_frames=24)
    path = tmp_path / "session.jsonl"
    rp.write_pose_log(path, log, (1280, 720))
    recs, display = rp.read_pose_log(path)
    assert display == (1280, 720) and len(recs) == 24
    a = rp.replay(scene, recs, display, stride=5, out_dir=tmp_path / "a", keep_gt=True)
    b = rp.replay(scene, recs, display, stride=5, out_dir=tmp_path / "b")
    assert [f.i for f in a] == [0, 5, 10, 15, 20]
    for fa, fb, r in zip(a, b, [recs[k] for k in (0, 5, 10, 15, 20)]):
        assert fa.jpeg == fb.jpeg and fa.ssim == fb.ssim and fa.psnr == fb.psnr
        assert (tmp_path / "a" / f"{r.i:06d}_gt.png").read_bytes() == (tmp_path / "b" / f"{r.i:06d}_gt.png").read_bytes()
        # the transmitted JPEG: the oracle's file of the same render at the logged profile
        low = tg.render(scene, r.pose, r.intr, r.width, r.height)
        assert fa.jpeg == ojpeg.encode(low, r.quality, restart=2)
        assert (tmp_path / "a" / f"{r.i:06d}_original.jpg").read_bytes() == fa.jpeg
        # the ground truth: a direct render at the display size, losslessly stored
        k = r.intr
        gt = tg.render(scene, r.pose, (k[0] * 1280 / r.width, k[1] * 720 / r.height, k[2] * 1280 / r.width,
                                       k[3] * 720 / r.height), 1280, 720)
        assert np.array_equal(fa.gt, gt)
        assert np.array_equal(_png_pixels((tmp_path / "a" / f"{r.i:06d}_gt.png").read_bytes()), gt)
        # metrics against the oracle
        up = oq.resample(low, 1280, 720)
        assert abs(fa.ssim - oq.ssim(gt, up)) <= 1e-5
        want = oq.psnr(gt, up)
        assert (fa.psnr == want) if math.isinf(want) else abs(fa.psnr - want) < 1e-9
