"""The CUDA JPEG encoder against the JPEG oracle: byte-identical files.

Inputs are frames the renderer produces (the encoder's real input) and
synthetic patterns, at sizes that are not multiples of the 16x16 MCU, at the
qualities of Table 1 and with several restart intervals."""
import numpy as np
import pytest

import synth
from oracle import jpeg as ojpeg
from tests import jpeg_decode

torch = pytest.importorskip("torch")
import paper_2605_08699_b300 as tg  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    tg.load_library()
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def frames(cuda):
    s = synth.config_scene(1)
    out = {}
    with tg.scene_from(s) as h:
        for (w, hh) in [(320, 240), (97, 61), (480, 270), (17, 9)]:
            out[(w, hh)] = tg.render(h, synth.config_trajectory(1)[40], synth.default_intrinsics(w, hh), w, hh)
    return out


@pytest.mark.parametrize("quality", [10, 35, 65, 90])
@pytest.mark.parametrize("size", [(320, 240), (97, 61), (480, 270), (17, 9)])
def test_rendered_frames_match_the_oracle(frames, size, quality):
    img = frames[size]
    # restart intervals of up to 4 MCUs take the warp-per-interval coder, longer ones
    # the thread-per-interval coder: both must give the oracle's file
    for restart in (1, 3, 4, 5, 64):
        got = tg.jpeg_encode(img, quality, restart_mcus=restart)
        assert got == ojpeg.encode(img, quality, restart=restart)


@pytest.mark.parametrize("seed", [0, 1])
def test_noise_and_extremes_match_the_oracle(seed):
    rng = np.random.default_rng(seed)
    img = rng.integers(0, 256, (45, 70, 4), dtype=np.uint8)   # long codes, stuffing
    img[:8, :8, :3] = 255
    img[8:16, :8, :3] = 0
    for q in (1, 50, 100):
        for restart in (2, 7):   # noise: long codes, zero runs of 16+, 0xFF stuffing in both coders
            assert tg.jpeg_encode(img, q, restart_mcus=restart) == ojpeg.encode(img, q, restart=restart)


def test_device_in_and_out_and_decodes(cuda, frames):
    img = frames[(480, 270)]
    ref = ojpeg.encode(img, 90, restart=2)
    d_in = torch.from_numpy(img).to(cuda)
    d_out = torch.zeros(1 << 20, dtype=torch.uint8, device=cuda)
    n = tg.jpeg_encode(d_in, 90, restart_mcus=2, out=d_out)
    assert bytes(d_out[:n].cpu().numpy()) == ref
    dec = jpeg_decode.decode(ref)
    y0 = (img[..., :3].astype(np.float64) @ [0.299, 0.587, 0.114])
    y1 = np.clip(np.round(dec), 0, 255) @ [0.299, 0.587, 0.114]
    assert 10 * np.log10(255 ** 2 / np.mean((y0 - y1) ** 2)) > 30.0


def test_small_output_buffer_reports_the_length(cuda, frames):
    img = frames[(97, 61)]
    small = np.zeros(64, np.uint8)
    with pytest.raises(tg.TigasError) as e:
        tg.jpeg_encode(img, 65, restart_mcus=1, out=small)
    assert e.value.status == tg.ERR_OVERFLOW


def test_full_hd_frame_matches_the_oracle(cuda):
    s = synth.config_scene(3, n=1_000_000)
    W, H = 1920, 1080
    with tg.scene_from(s, storage=tg.STORAGE_FP16) as h:
        img = tg.render(h, synth.config_trajectory(3)[10], synth.default_intrinsics(W, H), W, H)
    for q in (65, 90):
        assert tg.jpeg_encode(img, q, restart_mcus=2) == ojpeg.encode(img, q, restart=2)


@pytest.mark.parametrize("u,v", [(7, 7), (4, 5), (0, 6), (3, 0)])
def test_long_zero_runs_match_the_oracle(u, v):
    """A single DCT basis pattern per 8x8 block: its coefficient follows a zero
    run of up to 62 (three ZRL codes before it in zig-zag order)."""
    y, x = np.mgrid[0:48, 0:64]
    f = np.cos((2 * (x % 8) + 1) * u * np.pi / 16) * np.cos((2 * (y % 8) + 1) * v * np.pi / 16)
    img = np.zeros((48, 64, 4), np.uint8)
    for c in range(3):
        img[..., c] = np.clip(np.round(128 + (60 - 15 * c) * f), 0, 255).astype(np.uint8)
    for q in (100, 90):
        for restart in (1, 2, 5):
            assert tg.jpeg_encode(img, q, restart_mcus=restart) == ojpeg.encode(img, q, restart=restart)
