"""Allocation failures injected on the host (tigas_debug_fail_alloc).

A failed request must report TIGAS_ERR_OOM with a message, affect no other
request, and leave the library able to render a correct frame next: the
errors a client shows in place of the frame (Sec. 5.3 "Viewport Display")
and the isolation of stateless per-frame requests (Sec. 4.2).  The failures
are made on the host: the library's allocation wrapper returns
cudaErrorMemoryAllocation without calling the allocator.  Nothing faults,
traps or hangs the GPU.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2605_08699_b300 as tg  # noqa: E402

W, H = 160, 120
K = synth.default_intrinsics(W, H)


@pytest.fixture(scope="module")
def cuda():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    tg.load_library()
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def scene():
    return synth.config_scene(1, n=30_000)


@pytest.fixture(autouse=True)
def _clear_injection():
    yield
    tg.debug_fail_alloc(tg.DEVICE_ALLOC, 0)
    tg.debug_fail_alloc(tg.PINNED_ALLOC, 0)


def _expect_oom(fn):
    with pytest.raises(tg.TigasError) as e:
        fn()
    assert e.value.status == tg.ERR_OOM, e.value
    assert "alloc" in str(e.value) or "memory" in str(e.value)
    return str(e.value)


@pytest.mark.parametrize("on_device", [False, True])
def test_scene_load_reports_oom_and_the_next_load_renders(cuda, scene, on_device):
    arrs = [scene.means, scene.log_scales, scene.quats, scene.opacity_logits, scene.sh]
    if on_device:
        arrs = [torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(cuda) for a in arrs]
    with tg.scene_from(scene) as ref_h:
        want = tg.render(ref_h, synth.BASE_POSE, K, W, H)
    # host inputs: the first device allocation is the upload staging; device inputs: the scene itself
    tg.debug_fail_alloc(tg.DEVICE_ALLOC, 1, 1)
    _expect_oom(lambda: tg.scene_load(*arrs, sh_degree=scene.sh_degree))
    h = tg.scene_load(*arrs, sh_degree=scene.sh_degree)
    try:
        assert np.array_equal(tg.render(h, synth.BASE_POSE, K, W, H), want)
    finally:
        h.free()


def _render_dev(h, pose, out):
    tg.render(h, pose, K, W, H, out=out)   # device output: no host staging buffer is allocated
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_first_render_after_workspace_release_reports_oom_and_recovers(cuda, scene):
    out = torch.empty((H, W, 4), dtype=torch.uint8, device=cuda)
    with tg.scene_from(scene) as h:
        want = _render_dev(h, synth.BASE_POSE, out)
        # idle contexts dropped: the next render grows a fresh per-entry arena (both of
        # its attempts, with and without headroom, fail)
        tg.release_workspace()
        tg.debug_fail_alloc(tg.DEVICE_ALLOC, 1, 2)
        msg = _expect_oom(lambda: _render_dev(h, synth.BASE_POSE, out))
        assert "workspace" in msg
        tg.debug_fail_alloc(tg.DEVICE_ALLOC, 0)
        assert np.array_equal(_render_dev(h, synth.BASE_POSE, out), want)
        # a later allocation of the same launch set: the first slice's pair arena
        tg.release_workspace()
        tg.debug_fail_alloc(tg.DEVICE_ALLOC, 2, 2)
        _expect_oom(lambda: _render_dev(h, synth.BASE_POSE, out))
        tg.debug_fail_alloc(tg.DEVICE_ALLOC, 0)
        for _ in range(3):   # exact, captured, replayed
            assert np.array_equal(_render_dev(h, synth.BASE_POSE, out), want)


def test_pinned_host_allocation_failure_reports_oom_and_recovers(cuda, scene):
    out = torch.empty((H, W, 4), dtype=torch.uint8, device=cuda)
    with tg.scene_from(scene) as h:
        want = _render_dev(h, synth.BASE_POSE, out)
        tg.release_workspace()
        tg.debug_fail_alloc(tg.PINNED_ALLOC, 1, 1)   # a new render context's pinned read-back buffers
        _expect_oom(lambda: _render_dev(h, synth.BASE_POSE, out))
        assert np.array_equal(_render_dev(h, synth.BASE_POSE, out), want)


def test_server_batch_with_oom_fails_every_ticket_and_the_next_batch_is_correct(cuda, scene):
    tr = synth.trajectory(41, 8)
    with tg.scene_from(scene) as h:
        refs = [tg.render(h, p, K, W, H) for p in tr]
        # one slot; a long window so that the four requests form one launch set
        with tg.Server(max_batch=4, max_inflight=1, batch_window_us=500_000) as srv:
            tg.release_workspace()
            tg.debug_fail_alloc(tg.DEVICE_ALLOC, 1, 2)
            bufs = {}
            for i in range(4):
                b = torch.zeros((H, W, 4), dtype=torch.uint8, device=cuda)
                bufs[srv.submit(h, tr[i], K, W, H, b, client_id=i)] = (b, i)
            done = []
            while len(done) < 4:
                done += srv.poll(16, timeout_us=2_000_000)
            assert len({(c.admit_us, c.done_us) for c in done}) == 1   # one launch set
            assert all(c.status == tg.ERR_OOM for c in done)
            tg.debug_fail_alloc(tg.DEVICE_ALLOC, 0)
            bufs = {}
            for i in range(4, 8):
                b = torch.zeros((H, W, 4), dtype=torch.uint8, device=cuda)
                bufs[srv.submit(h, tr[i], K, W, H, b, client_id=i)] = (b, i)
            done = []
            while len(done) < 4:
                done += srv.poll(16, timeout_us=2_000_000)
            assert all(c.status == tg.OK for c in done)
            for c in done:
                b, i = bufs[c.ticket]
                assert np.array_equal(b.cpu().numpy(), refs[i])
