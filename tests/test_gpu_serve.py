"""The continuous-batching server: every camera's masks in the mix equal
what the same camera gives alone, also when cameras join and leave a running
server; admission refuses cameras that do not fit in free device memory."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.fixture(scope="module")
def cog():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1705_09339_gb300 import cog
    return cog


CAMS = [(160, 120, 3, "f16"), (320, 240, 5, "f16"), (640, 480, 5, "f16"), (97, 61, 3, "f32"), (200, 150, 5, "bf16")]


def test_each_camera_same_alone_and_in_the_mix(cog):
    import random
    import time

    from cogsynth import Scene
    from cogsynth.gpu import GpuScene
    from paper_1705_09339_gb300.serve import FrameServer
    NT, NF = 30, 14
    srv = FrameServer(reserve_bytes=1 << 30, keep_masks=True)
    data = []
    for i, (w, h, k, dt) in enumerate(CAMS):
        sc = Scene(w, h, 900 + i, kind="dynamic", n_train=NT, fg_frac=0.05, switch_at=4)
        gs = GpuScene(sc)
        tr = gs.render(0, NT)
        te = gs.render(NT, NF)
        cam = srv.admit(w, h, k, dt, tr)
        assert cam is not None
        data.append((cam, tr, [te[j].cpu().pin_memory() for j in range(NF)]))
    srv.start()
    # frames of all cameras arrive interleaved at random moments
    order = [(i, j) for i in range(len(CAMS)) for j in range(NF)]
    order.sort(key=lambda x: (x[1] + random.Random(x[0] * 100 + x[1]).random(), x[0]))
    for i, j in order:
        srv.submit(data[i][0], data[i][2][j])
        if j % 3 == 0:
            time.sleep(0.001)
    stats = srv.stop()
    assert stats["frames"] == len(CAMS) * NF and stats["latency_ms"]["p99"] > 0
    for i, (w, h, k, dt) in enumerate(CAMS):
        cam, tr, frames = data[i]
        got = sorted(srv.results[cam.id], key=lambda x: x[0])
        assert [s for s, _ in got] == list(range(NF))
        p = cog.cog_default_params(w, h, k, state_dtype=dt)
        c = cog.cog_create(p, torch.cuda.current_stream().cuda_stream)
        cog.cog_train_prior(c, tr, NT)
        m = torch.empty((h, w), dtype=torch.uint8, device="cuda")
        for j in range(NF):
            cog.cog_apply(c, frames[j].cuda(), m)
            assert np.array_equal(m.cpu().numpy(), got[j][1]), (i, j)
        cog.cog_destroy(c)
    srv.close()


def test_admission_by_free_memory(cog):
    from paper_1705_09339_gb300.serve import FrameServer
    free, total = torch.cuda.mem_get_info()
    srv = FrameServer(reserve_bytes=free)          # nothing fits above this reserve
    tr = torch.zeros((2, 48, 64, 3), dtype=torch.uint8, device="cuda")
    assert srv.admit(64, 48, 3, "f16", tr) is None
    assert len(srv.refused) == 1
    srv.close()


def test_camera_joins_a_running_server(cog):
    # two cameras serve; a third is admitted and trained while frames of the
    # first two are on the GPU, joins between steps, and every camera's
    # masks still equal what it gives alone
    import time

    from cogsynth import Scene
    from cogsynth.gpu import GpuScene
    from paper_1705_09339_gb300.serve import FrameServer
    NT, NF = 30, 12
    cams = [(160, 120, 3, "f16"), (97, 61, 5, "f32"), (200, 150, 5, "bf16")]
    srv = FrameServer(reserve_bytes=1 << 30, keep_masks=True)
    data = []
    for i, (w, h, k, dt) in enumerate(cams):
        sc = Scene(w, h, 700 + i, kind="dynamic", n_train=NT, fg_frac=0.05, switch_at=4)
        gs = GpuScene(sc)
        data.append((gs.render(0, NT), [f.cpu().pin_memory() for f in gs.render(NT, NF)]))
    handles = [srv.admit(*cams[i], data[i][0]) for i in range(2)]
    assert all(c is not None for c in handles)
    srv.start()
    for j in range(NF // 2):
        for i in range(2):
            srv.submit(handles[i], data[i][1][j])
    late = srv.admit(*cams[2], data[2][0])          # joins while the first frames run
    assert late is not None and late.id == 2
    handles.append(late)
    with pytest.raises(cog.CogError):
        cog.cog_server_add(srv.srv, late.ctx)       # already a stream of the server
    for j in range(NF):
        if j >= NF // 2:
            for i in range(2):
                srv.submit(handles[i], data[i][1][j])
        srv.submit(late, data[2][1][j])
        time.sleep(0.0005)
    stats = srv.stop()
    assert stats["frames"] == 3 * NF and stats["cameras"] == 3
    for i, (w, h, k, dt) in enumerate(cams):
        got = sorted(srv.results[handles[i].id], key=lambda x: x[0])
        assert [s for s, _ in got] == list(range(NF))
        p = cog.cog_default_params(w, h, k, state_dtype=dt)
        c = cog.cog_create(p, torch.cuda.current_stream().cuda_stream)
        cog.cog_train_prior(c, data[i][0], NT)
        m = torch.empty((h, w), dtype=torch.uint8, device="cuda")
        for j in range(NF):
            cog.cog_apply(c, data[i][1][j].cuda(), m)
            assert np.array_equal(m.cpu().numpy(), got[j][1]), (i, j)
        cog.cog_destroy(c)
    srv.close()


def test_camera_leaves_and_its_index_is_reused(cog):
    # three cameras serve; the second leaves while its frames are on the GPU:
    # every frame it was given is still completed, its index refuses frames
    # until a fourth camera joins and takes it, and every camera's masks
    # equal what it gives alone
    from cogsynth import Scene
    from cogsynth.gpu import GpuScene
    from paper_1705_09339_gb300.serve import FrameServer
    NT, NF = 30, 12
    cams = [(160, 120, 3, "f16"), (97, 61, 5, "f32"), (200, 150, 5, "bf16"), (64, 48, 3, "f16")]
    srv = FrameServer(reserve_bytes=1 << 30, keep_masks=True)
    data = []
    for i, (w, h, k, dt) in enumerate(cams):
        sc = Scene(w, h, 800 + i, kind="dynamic", n_train=NT, fg_frac=0.05, switch_at=5)
        gs = GpuScene(sc)
        data.append((gs.render(0, NT), [f.cpu().pin_memory() for f in gs.render(NT, NF)]))
    h = [srv.admit(*cams[i], data[i][0]) for i in range(3)]
    assert [c.id for c in h] == [0, 1, 2]
    srv.start()
    for j in range(NF // 2):
        for i in range(3):
            srv.submit(h[i], data[i][1][j])
    free_before = torch.cuda.mem_get_info()[0]
    srv.leave(h[1])
    assert len(h[1].masks) == NF // 2 and torch.cuda.mem_get_info()[0] > free_before
    with pytest.raises(cog.CogError):
        cog.cog_server_submit(srv.srv, 1, data[1][1][0], np.empty((61, 97), np.uint8))
    with pytest.raises(cog.CogError):
        cog.cog_server_remove(srv.srv, 1)          # already left
    with pytest.raises(cog.CogError):
        cog.cog_server_remove(srv.srv, 7)          # no such camera
    late = srv.admit(*cams[3], data[3][0])
    assert late is not None and late.id == 1       # the freed index
    for j in range(NF):
        if j >= NF // 2:
            for i in (0, 2):
                srv.submit(h[i], data[i][1][j])
        srv.submit(late, data[3][1][j])
    stats = srv.stop()
    assert stats["frames"] == 3 * NF + NF // 2 and stats["cameras"] == 3
    for i, cam in ((0, h[0]), (1, h[1]), (2, h[2]), (3, late)):
        w, hh, k, dt = cams[i]
        got = sorted(cam.masks, key=lambda x: x[0])
        n = len(got)
        assert [s for s, _ in got] == list(range(n)) and n == (NF // 2 if i == 1 else NF)
        p = cog.cog_default_params(w, hh, k, state_dtype=dt)
        c = cog.cog_create(p, torch.cuda.current_stream().cuda_stream)
        cog.cog_train_prior(c, data[i][0], NT)
        m = torch.empty((hh, w), dtype=torch.uint8, device="cuda")
        for j in range(n):
            cog.cog_apply(c, data[i][1][j].cuda(), m)
            assert np.array_equal(m.cpu().numpy(), got[j][1]), (i, j)
        cog.cog_destroy(c)
    srv.close()


def test_last_camera_cannot_leave(cog):
    from paper_1705_09339_gb300.serve import FrameServer
    srv = FrameServer(reserve_bytes=1 << 30)
    tr = torch.zeros((2, 48, 64, 3), dtype=torch.uint8, device="cuda")
    cam = srv.admit(64, 48, 3, "f16", tr)
    srv.start()
    with pytest.raises(cog.CogError) as e:
        cog.cog_server_remove(srv.srv, cam.id)
    assert e.value.status == cog.COG_ERR_INVALID_ARG
    # the camera still serves
    f = torch.zeros((48, 64, 3), dtype=torch.uint8).pin_memory()
    srv.submit(cam, f)
    assert srv.stop()["frames"] == 1
    srv.close()
