"""CUDA path vs FP64 oracle, element by element, through the C ABI.

Bars (FP32 state): masks and stage maps bit-identical on every pixel whose
decision history never came within 1e-4 relative of a threshold (the
oracle's near record); overall mask agreement >= 99.99 %; model means,
variances, weights and confidence within 1e-4 relative (denominator
max(|x|, 1)) on never-near pixels; integer work (prior, residue weights,
previous frame, labels) bit-exact.
"""
import numpy as np
import pytest

from cog_harness import (GpuRun, compare_stream, oracle_run, oracle_state, params, random_frame,
                         random_state, set_oracle_state, state_errors)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


# ------------------------------------------------------------- generator
@pytest.mark.parametrize("kind", ["rects", "dynamic"])
def test_generator_twin_bit_exact(kind):
    from cogsynth import Scene
    from cogsynth.gpu import GpuScene
    sc = Scene(203, 77, 9, kind=kind, n_train=5, fg_frac=0.08, switch_at=3)
    g, gt = GpuScene(sc).render(0, 12, gt=True)
    for t in range(12):
        f, m = sc.render(t)
        assert np.array_equal(g[t].cpu().numpy().reshape(-1, 3), f)
        assert np.array_equal(gt[t].cpu().numpy().reshape(-1), m)


# -------------------------------------------------------------- training
@pytest.mark.parametrize("bw", [1, 7])
def test_prior_parity_other_bandwidths(bw):
    # bandwidths other than 4 take the prior kernel's bounds-checked taps
    from cogsynth import Scene
    W, H, N = 37, 29, 23
    sc = Scene(W, H, 5, kind="dynamic", n_train=N, fg_frac=0.05)
    fr, _ = sc.frames(0, N)
    d = params(W, H, 3, kde_bw=bw)
    g = GpuRun(d)
    g.train(fr)
    gs = g.state()
    g.close()
    o = oracle_run(d)
    o.train(fr)
    assert np.array_equal(gs["kde"], oracle_state(o)["kde"])


@pytest.mark.parametrize("W,H,K,N", [(160, 120, 3, 200), (37, 29, 5, 17), (1, 1, 1, 2), (91, 45, 8, 40)])
def test_training_parity(W, H, K, N):
    from cogsynth import Scene
    sc = Scene(W, H, 3, kind="dynamic", n_train=N, fg_frac=0.05)
    fr, _ = sc.frames(0, N)
    d = params(W, H, K)
    g = GpuRun(d)
    g.train(fr)
    gs = g.state()
    g.close()
    o = oracle_run(d)
    near0 = o.train(fr, want_near=True)
    os_ = oracle_state(o)
    assert np.array_equal(gs["kde"], os_["kde"])
    assert np.array_equal(gs["qa"], os_["qa"]) and np.array_equal(gs["qb"], os_["qb"])
    assert np.array_equal(gs["prev"], os_["prev"])
    assert (gs["conf"] == 0.5).all()
    # the warm-up runs N-1 mixture steps: labels and state may differ only
    # on pixels where one of its decisions came near a threshold
    ok = near0 == 0
    assert np.array_equal(gs["label"][ok], os_["label"][ok])
    e = state_errors(gs, os_, ok)
    for k in ("w", "mu", "var", "rga_m", "rga_v"):
        assert e[k] < TOL, (k, e[k])


# ----------------------------------------------------- free-running stream
def _stream(W, H, K, NT, NF, kind, dtype="f32", flags=15, seed=1, fg=0.03, switch_at=10**6):
    from cogsynth import Scene
    sc = Scene(W, H, seed, kind=kind, n_train=NT, fg_frac=fg, switch_at=switch_at)
    fr, _ = sc.frames(0, NT + NF)
    d = params(W, H, K, flags=flags)
    g = GpuRun(d, dtype)
    g.train(fr[:NT])
    gm, gsm, gst = g.apply(fr[NT:])
    gstate = g.state()
    g.close()
    o = oracle_run(d)
    near0 = o.train(fr[:NT], want_near=True)
    om, osm, near, ost = [], [], [], []
    for t in range(NF):
        m, s, n, st = o.apply(fr[NT + t])
        om.append(m); osm.append(s); near.append(n); ost.append(st)
    near[0] = near[0] | near0   # warm-up decisions near a threshold count too
    return (gm, gsm, gst, gstate), (np.stack(om), np.stack(osm), np.stack(near), ost, oracle_state(o))


def test_qvga_stream_fp32_matches_oracle():
    # the 160x120 workload: 200 training frames, 300 test frames, K=3, FP32
    (gm, gsm, gst, gs), (om, osm, near, ost, os_) = _stream(160, 120, 3, 200, 300, "rects")
    agree, unexplained, ever = compare_stream(gm, gsm, om, osm, near)
    assert unexplained == 0
    assert agree >= 0.9999
    e = state_errors(gs, os_, ~ever)
    for k in ("w", "mu", "var", "rga_m", "rga_v", "conf"):
        assert e[k] <= TOL, (k, e[k])
    for k in ("label", "prev", "qa", "qb"):
        assert e[k] == 0, k
    # per-frame stage occupancy equals the oracle's up to near-threshold pixels
    for t in range(len(ost)):
        diff = sum(abs(a - b) for a, b in zip(gst[t]["n_stage"], ost[t]["n_stage"]))
        assert diff <= 2 * int((gsm[t] != osm[t]).sum()), t
        assert gst[t]["illum_flag"] == ost[t]["illum_flag"]


@pytest.mark.parametrize("W,H", [(37, 29), (1, 1), (1023, 1), (1025, 3), (129, 64)])
def test_ragged_sizes_match_oracle(W, H):
    # sizes that are not multiples of the 8-pixel thread group or the
    # 1024-pixel tile, single pixels, and a tile plus one
    (gm, gsm, gst, gs), (om, osm, near, ost, os_) = _stream(W, H, 3, 30, 40, "dynamic", fg=0.1,
                                                             switch_at=20, seed=5)
    agree, unexplained, ever = compare_stream(gm, gsm, om, osm, near)
    assert unexplained == 0
    e = state_errors(gs, os_, ~ever)
    for k in ("w", "mu", "var", "rga_m", "rga_v", "conf"):
        assert e[k] <= TOL, (k, e[k])


def test_vga_dynamic_stream_with_light_switch():
    # the 640x480 dynamic-background workload (K=5) over a window of frames
    # that contains the +60 light switch: the illumination counter must flag
    # the frame after the switch on both sides
    (gm, gsm, gst, gs), (om, osm, near, ost, os_) = _stream(640, 480, 5, 100, 40, "dynamic", seed=2,
                                                             fg=0.03, switch_at=20)
    agree, unexplained, ever = compare_stream(gm, gsm, om, osm, near)
    assert unexplained == 0
    assert agree >= 0.9999
    flags_g = [s["illum_flag"] for s in gst]
    flags_o = [s["illum_flag"] for s in ost]
    assert flags_g == flags_o
    assert flags_o[21] == 1
    e = state_errors(gs, os_, ~ever)
    for k in ("w", "mu", "var", "rga_m", "rga_v", "conf"):
        assert e[k] <= TOL, (k, e[k])


def test_temporal_sampling_stream_matches_oracle():
    # confidence-based temporal sampling on: saturated pixels are looked at
    # every 4 frames in 64-pixel phase blocks; both sides must skip the same
    # pixels on the same frames
    (gm, gsm, gst, gs), (om, osm, near, ost, os_) = _stream(160, 120, 3, 200, 120, "rects", flags=31)
    agree, unexplained, ever = compare_stream(gm, gsm, om, osm, near)
    assert unexplained == 0
    assert agree >= 0.9999
    skipped = sum(s["n_stage"][5] for s in ost)
    assert skipped > 0.2 * 160 * 120 * 120          # sampling really engages
    assert sum(s["n_stage"][5] for s in gst) == pytest.approx(skipped, rel=1e-3)
    e = state_errors(gs, os_, ~ever)
    for k in ("w", "mu", "var", "rga_m", "rga_v", "conf"):
        assert e[k] <= TOL, (k, e[k])


# --------------------------------------------------- seeded random states
@pytest.mark.parametrize("K", [1, 3, 5, 8])
@pytest.mark.parametrize("flags", [15, 0, 1 | 2, 4 | 8, 15 | 32, 2 | 32, 15 | 64, 64])
def test_seeded_state_steps_match_oracle(K, flags):
    rng = np.random.default_rng(100 + K * 16 + flags)
    W, H = 53, 41
    P = W * H
    d = params(W, H, K, flags=flags)
    st = random_state(rng, P, K, mode1=bool(flags & 32), perchan=bool(flags & 64))
    g = GpuRun(d)
    g.train(np.zeros((2, P, 3), np.uint8))
    g.set_state(st)
    o = oracle_run(d)
    set_oracle_state(o, st)
    ever = np.zeros(P, bool)
    for step in range(6):
        f = random_frame(rng, st)
        gm, gsm, gst = g.apply(f[None])
        om, osm, near, ost = o.apply(f)
        ever |= near != 0
        bad = (gm[0] != om) | (gsm[0] != osm)
        assert not (bad & ~ever).any(), (step, np.nonzero(bad & ~ever)[0][:10])
        assert gst[0]["illum_flag"] == ost["illum_flag"]
    gst = g.state()
    e = state_errors(gst, oracle_state(o), ~ever)
    g.close()
    for k in ("w", "mu", "var", "rga_m", "rga_v", "conf", "wc"):
        if k in e:
            assert e[k] <= TOL, (k, e[k])
    assert e["label"] == 0 and e["prev"] == 0
    if flags & 32:
        assert np.array_equal(gst["top"][~ever], o.state.top[~ever])


@pytest.mark.parametrize("dtype,tol", [("f16", 2e-3), ("bf16", 1.6e-2)])
def test_seeded_state_16bit_storage(dtype, tol):
    # 16-bit storage rounds every stored value: one step from an identical
    # start agrees with the FP64 oracle to the storage precision
    rng = np.random.default_rng(7)
    W, H, K = 64, 32, 5
    P = W * H
    d = params(W, H, K)
    st = random_state(rng, P, K, dtype)
    g = GpuRun(d, dtype)
    g.train(np.zeros((2, P, 3), np.uint8))
    g.set_state(st)
    o = oracle_run(d)
    set_oracle_state(o, st)
    f = random_frame(rng, st)
    gm, gsm, _ = g.apply(f[None])
    om, osm, near, _ = o.apply(f)
    ok = near == 0
    assert (gm[0][ok] == om[ok]).mean() >= 0.999
    e = state_errors(g.state(), oracle_state(o), ok & (gm[0] == om) & (gsm[0] == osm))
    g.close()
    for k in ("w", "mu", "var", "rga_m", "rga_v", "conf"):
        assert e[k] <= tol, (k, e[k])


# --------------------------------------------- cascade off == plain mixture
@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
def test_cascade_off_equals_plain_gmm_kernel(dtype):
    from cogsynth import Scene
    W, H, K = 97, 61, 5
    sc = Scene(W, H, 8, kind="dynamic", n_train=40, fg_frac=0.08, switch_at=15)
    fr, _ = sc.frames(0, 80)
    d = params(W, H, K, flags=0)
    a, b = GpuRun(d, dtype), GpuRun(d, dtype)
    a.train(fr[:40])
    b.train(fr[:40])
    ma, _, _ = a.apply(fr[40:])
    mb, _, _ = b.apply(fr[40:], plain=True)
    sa, sb = a.state(), b.state()
    a.close(), b.close()
    assert np.array_equal(ma, mb)
    for k in ("w", "mu", "var"):
        assert np.array_equal(sa[k], sb[k]), k


def test_plain_gmm_kernel_matches_oracle():
    from cogsynth import Scene
    W, H, K = 120, 90, 3
    sc = Scene(W, H, 12, kind="dynamic", n_train=50, fg_frac=0.05, switch_at=10)
    fr, _ = sc.frames(0, 110)
    d = params(W, H, K, flags=0)
    g = GpuRun(d)
    g.train(fr[:50])
    gm, _, _ = g.apply(fr[50:], plain=True)
    gs = g.state()
    g.close()
    o = oracle_run(d)
    ever = o.train(fr[:50], want_near=True) != 0
    for t in range(60):
        m, _, n, _ = o.apply(fr[50 + t])
        ever |= n != 0
        assert not ((gm[t] != m) & ~ever).any(), t
    e = state_errors(gs, oracle_state(o), ~ever)
    for k in ("w", "mu", "var"):
        assert e[k] <= TOL, (k, e[k])


# ------------------------------------------------------------ ABI behaviour
def test_abi_errors_and_state_roundtrip():
    from cogsynth import Scene
    from paper_1705_09339_gb300 import cog
    W, H, K = 64, 40, 3
    d = params(W, H, K)
    g = GpuRun(d)
    f = torch.zeros((H, W, 3), dtype=torch.uint8, device="cuda")
    m = torch.zeros((H, W), dtype=torch.uint8, device="cuda")
    with pytest.raises(cog.CogError) as e:
        cog.cog_apply(g.ctx, f, m)
    assert e.value.status == cog.COG_ERR_STATE
    sc = Scene(W, H, 2, kind="dynamic", n_train=20, fg_frac=0.1, switch_at=5)
    fr, _ = sc.frames(0, 40)
    g.train(fr[:20])
    with pytest.raises(cog.CogError) as e:
        cog.cog_train_prior(g.ctx, g._dev_frames(fr[:1]), 1)
    assert e.value.status == cog.COG_ERR_INVALID_ARG
    g.apply(fr[20:25])
    snap = cog.cog_export_state(g.ctx, g.p)
    m1, s1, st1 = g.apply(fr[25:40])
    h = GpuRun(d)
    cog.cog_import_state(h.ctx, snap)
    m2, s2, st2 = h.apply(fr[25:40])
    assert np.array_equal(m1, m2) and np.array_equal(s1, s2) and st1 == st2
    last, total = cog.cog_read_stats(h.ctx)
    assert total["frame"] == 20 and last == st2[-1]
    g.close(), h.close()


def test_unaligned_frames_and_masks_give_identical_results():
    # frames at every byte offset mod 16 (no TMA staging) and masks at odd
    # offsets (no vector stores) must give what aligned buffers give
    from cogsynth import Scene
    W, H, K = 75, 41, 3
    sc = Scene(W, H, 13, kind="dynamic", n_train=20, fg_frac=0.1, switch_at=3)
    fr, _ = sc.frames(0, 36)
    d = params(W, H, K)
    a, b = GpuRun(d), GpuRun(d)
    a.train(fr[:20])
    b.train(fr[:20])
    ma, sa, _ = a.apply(fr[20:])
    P = W * H
    raw = torch.zeros(16 * P * 3 + 64, dtype=torch.uint8, device="cuda")
    mraw = torch.zeros(16 * (P + 8) + 64, dtype=torch.uint8, device="cuda")
    from paper_1705_09339_gb300 import cog
    mb = np.zeros_like(ma)
    for i in range(16):
        off = (i * 7) % 16
        f = raw[off + i * P * 3: off + (i + 1) * P * 3]
        f.copy_(torch.from_numpy(fr[20 + i].reshape(-1)).cuda())
        m = mraw[1 + i * (P + 8): 1 + i * (P + 8) + P]
        cog.cog_apply(b.ctx, f, m)
        mb[i] = m.cpu().numpy()
    a.close(), b.close()
    assert np.array_equal(ma, mb)


def test_caller_owned_state_and_host_buffers():
    from cogsynth import Scene
    from paper_1705_09339_gb300 import cog
    W, H, K = 80, 48, 3
    sc = Scene(W, H, 6, kind="rects", n_train=30)
    fr, _ = sc.frames(0, 40)
    d = params(W, H, K)
    p = GpuRun(d).p
    buf = torch.empty(cog.cog_state_bytes(p), dtype=torch.uint8, device="cuda")
    ctx = cog.cog_create(p, torch.cuda.current_stream().cuda_stream, buf)
    frt = torch.from_numpy(fr.reshape(40, H, W, 3)).cuda()
    cog.cog_train_prior(ctx, frt[:30], 30)
    ref = GpuRun(d)
    ref.train(fr[:30])
    rm, _, _ = ref.apply(fr[30:])
    masks = np.zeros((10, W * H), np.uint8)
    for i in range(10):
        cog.cog_apply_host(ctx, np.ascontiguousarray(fr[30 + i]), masks[i])
    assert np.array_equal(masks, rm)
    n, ptr = cog.cog_info(ctx)
    assert n == 10 and ptr == buf.data_ptr()
    cog.cog_destroy(ctx)
    ref.close()


@pytest.mark.parametrize("pinned", [True, False, "registered"])
def test_host_frames_pipeline_equals_device_apply(pinned):
    # cog_apply_host_frames overlaps uploads and downloads with the kernels
    # through two device slots; results must equal cog_apply on device
    # buffers frame by frame (also with a light switch inside the run)
    from cogsynth import Scene
    from paper_1705_09339_gb300 import cog
    W, H, K, NT, NF = 320, 240, 5, 40, 37
    sc = Scene(W, H, 7, kind="dynamic", n_train=NT, fg_frac=0.05, switch_at=20)
    fr, _ = sc.frames(0, NT + NF)
    d = params(W, H, K)
    ref = GpuRun(d, "f16")
    ref.train(fr[:NT])
    rm, _, _ = ref.apply(fr[NT:])
    g = GpuRun(d, "f16")
    g.train(fr[:NT])
    host = torch.from_numpy(np.ascontiguousarray(fr[NT:]).reshape(NF, H, W, 3))
    masks = torch.zeros((NF, H, W), dtype=torch.uint8)
    blocks = []
    if pinned == "registered":
        # frames and masks in cog_host_alloc memory (huge pages locked with
        # cudaHostRegister)
        import ctypes
        views = []
        for t in (host, masks):
            addr = cog.cog_host_alloc(t.numel())
            blocks.append(addr)
            a = np.ctypeslib.as_array(ctypes.cast(addr, ctypes.POINTER(ctypes.c_uint8)), shape=(t.numel(),))
            v = torch.from_numpy(a[:t.numel()]).view(t.shape)
            v.copy_(t)
            views.append(v)
        host, masks = views
    elif pinned:
        host, masks = host.pin_memory(), masks.pin_memory()
    cog.cog_apply_host_frames(g.ctx, host.numpy(), masks.numpy())
    assert np.array_equal(masks.numpy().reshape(NF, -1), rm)
    sa, sb = ref.state(), g.state()
    for k in sa:
        assert np.array_equal(sa[k], sb[k]), k
    # a second call continues the same stream
    cog.cog_apply_host_frames(g.ctx, host.numpy()[:5].copy(), masks.numpy()[:5].copy())
    assert cog.cog_info(g.ctx)[0] == NF + 5
    ref.close(); g.close()
    del host, masks
    for addr in blocks:
        cog.cog_host_free(addr)
    with pytest.raises(cog.CogError):
        cog.cog_host_free(blocks[0] if blocks else 8)   # freed already / never allocated


def test_mode1_stream_matches_oracle():
    # the Fig. 1 reading (stage 1 = the mixture's rank-1 mode, written back on
    # the transition) on the 160x120 workload, FP32
    W, H, K = 160, 120, 3
    (gm, gsm, gst, gs), (om, osm, near, ost, os_) = _stream(W, H, K, 200, 300, "rects", flags=15 | 32)
    agree, unexplained, ever = compare_stream(gm, gsm, om, osm, near)
    assert unexplained == 0 and agree >= 0.9999
    e = state_errors(gs, os_, ~ever)
    for k in ("w", "mu", "var", "rga_m", "rga_v", "conf"):
        assert e[k] <= TOL, (k, e[k])
    assert np.array_equal(gs["top"][~ever], os_["top"][~ever])


def test_perchan_stream_matches_oracle():
    # per-channel independent mixtures on the 160x120 workload, FP32
    W, H, K = 160, 120, 3
    (gm, gsm, gst, gs), (om, osm, near, ost, os_) = _stream(W, H, K, 200, 300, "rects", flags=15 | 64)
    agree, unexplained, ever = compare_stream(gm, gsm, om, osm, near)
    assert unexplained == 0 and agree >= 0.9999
    e = state_errors(gs, os_, ~ever)
    for k in ("wc", "mu", "var", "rga_m", "rga_v", "conf"):
        assert e[k] <= TOL, (k, e[k])


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_perchan_on_gray_input_equals_shared_weights_on_the_gpu(dtype):
    # R = G = B: the per-channel kernels must reproduce the shared-weight
    # kernels bit for bit (masks, stage maps, means, variances; each
    # channel's weights equal to the shared weights)
    from cogsynth import Scene
    W, H, K, NT, NF = 96, 64, 5, 30, 40
    sc = Scene(W, H, 23, kind="dynamic", n_train=NT, fg_frac=0.1, switch_at=20)
    fr, _ = sc.frames(0, NT + NF)
    gray = np.ascontiguousarray(np.repeat(fr[..., :1], 3, axis=-1))
    a = GpuRun(params(W, H, K), dtype)
    b = GpuRun(params(W, H, K, flags=15 | 64), dtype)
    a.train(gray[:NT])
    b.train(gray[:NT])
    am, asg, _ = a.apply(gray[NT:])
    bm, bsg, _ = b.apply(gray[NT:])
    assert np.array_equal(am, bm) and np.array_equal(asg, bsg)
    sa, sb = a.state(), b.state()
    assert np.array_equal(sa["mu"], sb["mu"]) and np.array_equal(sa["var"], sb["var"])
    for c in range(3):
        assert np.array_equal(sb["wc"][:, c, :], sa["w"])
    a.close(); b.close()


def test_plain_gmm_refused_with_perchan():
    from paper_1705_09339_gb300 import cog
    g = GpuRun(params(32, 16, 3, flags=15 | 64))
    g.train(np.zeros((2, 32 * 16, 3), np.uint8))
    f = torch.zeros((16, 32, 3), dtype=torch.uint8, device="cuda")
    m = torch.zeros((16, 32), dtype=torch.uint8, device="cuda")
    with pytest.raises(cog.CogError) as e:
        cog.cog_apply_plain_gmm(g.ctx, f, m)
    assert e.value.status == cog.COG_ERR_INVALID_ARG
    g.close()


def test_vga_full_workload_fp32_matches_oracle():
    # the whole 640x480 dynamic-background workload as specified: 500
    # training frames, 1000 test frames with the +60 light switch at test
    # frame 600, K=5, FP32 state, free-running against the FP64 oracle
    # (frames from the generator's GPU twin, bit-identical to its CPU side)
    from cogsynth import workload
    from cogsynth.gpu import GpuScene
    wl = workload("vga_dynamic", fg_frac=0.03)
    sc, K, NT, NF = wl["scene"], wl["K"], wl["n_train"], wl["n_test"]
    W, H = sc.width, sc.height
    fr = GpuScene(sc).render(0, NT + NF).cpu().numpy().reshape(NT + NF, W * H, 3)
    d = params(W, H, K)
    g = GpuRun(d, "f32")
    g.train(fr[:NT])
    gm, gsm, gst = g.apply(fr[NT:])
    gs = g.state()
    g.close()
    o = oracle_run(d)
    ever = o.train(fr[:NT], want_near=True) != 0
    unexplained = agree = 0
    flags_o = []
    for t in range(NF):
        m, s, near, st = o.apply(fr[NT + t])
        ever |= near != 0
        unexplained += int((((gm[t] != m) | (gsm[t] != s)) & ~ever).sum())
        agree += int((gm[t] == m).sum())
        flags_o.append(st["illum_flag"])
    assert unexplained == 0
    assert agree / gm.size >= 0.9999
    assert [s["illum_flag"] for s in gst] == flags_o
    assert flags_o[601] == 1
    e = state_errors(gs, oracle_state(o), ~ever)
    for k in ("w", "mu", "var", "rga_m", "rga_v", "conf"):
        assert e[k] <= TOL, (k, e[k])
    for k in ("label", "prev", "qa", "qb"):
        assert e[k] == 0, k
