"""Full-size parity in the benchmark's configuration: the 1920x1080 dynamic
stream, K=5, 500 training frames, FP32 and FP16 state, default launch
shape.  The oracle computes a sample of pixels one by one (pixels are
independent once the illumination counter, the only cross-pixel coupling, is
off), rendered by the CPU generator from the same counters."""
import numpy as np
import pytest

from cog_harness import params, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

W, H, K, NT, NF = 1920, 1080, 5, 500, 40


@pytest.fixture(scope="module")
def stream():
    import __graft_entry__
    __graft_entry__.build()
    from cogsynth import workload
    from cogsynth.gpu import GpuScene
    sc = workload("hd_dynamic", fg_frac=0.02)["scene"]
    gs = GpuScene(sc)
    rng = np.random.default_rng(11)
    P = W * H
    pix = np.unique(np.concatenate([rng.integers(0, P, 3800), [0, 1, 511, 512, 1023, 1024, P - 2, P - 1],
                                    np.arange(100) * 20736 + 3]))
    return sc, gs, pix


@pytest.mark.parametrize("dtype,bits", [("f32", 8), ("f16", 8), ("f16", 4)])
def test_full_size_sampled_pixels_match_oracle(stream, dtype, bits):
    # bits: the scene prior's width (kde_bits), 8 or 4
    import oracle
    from paper_1705_09339_gb300 import cog
    sc, gs, pix = stream
    flags = 1 | 2 | 4                       # FD | RGA | CONF (no illumination coupling)
    d = params(W, H, K, flags=flags, kde_bits=bits)
    p = cog.cog_default_params(W, H, K, state_dtype=dtype)
    for k, v in d.items():
        if k not in ("width", "height", "K"):
            setattr(p, "eta_conf" if k == "eta" else k, v)
    ctx = cog.cog_create(p, torch.cuda.current_stream().cuda_stream)
    tr = gs.render(0, NT)
    cog.cog_train_prior(ctx, tr, NT)
    del tr
    te = gs.render(NT, NF)
    pt = torch.from_numpy(pix).cuda()
    gm = np.zeros((NF, len(pix)), np.uint8)
    m = torch.empty((H, W), dtype=torch.uint8, device="cuda")
    for i in range(NF):
        cog.cog_apply(ctx, te[i], m)
        gm[i] = m.reshape(-1)[pt].cpu().numpy()
    gs_state = cog.decode_state(cog.cog_export_state(ctx, p), p)
    cog.cog_destroy(ctx)

    od = dict(d, width=len(pix), height=1)
    o = oracle.Oracle(od)
    trs = np.stack([sc.render(t, pix)[0] for t in range(NT)])
    ever = o.train(trs, want_near=True) != 0   # warm-up decisions near a threshold
    bad = 0
    agree = 0
    for i in range(NF):
        f, _ = sc.render(NT + i, pix)
        om, _, near, _ = o.apply(f)
        ever |= near != 0
        bad += int(((gm[i] != om) & ~ever).sum())
        agree += int((gm[i] == om).sum())
    frac = agree / (NF * len(pix))
    if dtype == "f32":
        assert bad == 0
        assert frac >= 0.9999
        ok = ~ever
        for k in ("w", "mu", "var", "rga_m", "rga_v", "conf"):
            e = rel_err(gs_state[k][pix][ok], getattr(o.state, k)[ok]).max()
            assert e <= 1e-4, (k, e)
    else:
        # 16-bit storage: agreement with the FP64 oracle, stated per config
        assert frac >= 0.995, frac


def test_full_size_with_illumination_counter_teacher_forced():
    # the same stream with the illumination counter on and a +60 light
    # switch at test frame 20.  The counter is the one cross-pixel coupling
    # (a frame is flagged when more than 70 % of the previous frame's pixels
    # reached the mixture stage), which a pixel sample cannot recompute: the
    # GPU's whole-frame counts decide each frame's flag, and the oracle is
    # handed that flag (teacher-forced) while it computes every sampled pixel
    # itself; the masks it then gives must be the GPU's away from
    # near-threshold decisions, the flagged frame included.
    import oracle
    from cogsynth import Scene
    from cogsynth.gpu import GpuScene
    from paper_1705_09339_gb300 import cog
    NF2 = 30
    sc = Scene(W, H, 3, kind="dynamic", n_train=NT, fg_frac=0.02, switch_at=20)
    gs = GpuScene(sc)
    P = W * H
    pix = np.unique(np.random.default_rng(12).integers(0, P, 3000))
    d = params(W, H, K)                      # FD | RGA | CONF | ILLUM
    p = cog.cog_default_params(W, H, K, state_dtype="f32")
    for k, v in d.items():
        if k not in ("width", "height", "K"):
            setattr(p, "eta_conf" if k == "eta" else k, v)
    ctx = cog.cog_create(p, torch.cuda.current_stream().cuda_stream)
    tr = gs.render(0, NT)
    cog.cog_train_prior(ctx, tr, NT)
    del tr
    te = gs.render(NT, NF2)
    pt = torch.from_numpy(pix).cuda()
    gm = np.zeros((NF2, len(pix)), np.uint8)
    m = torch.empty((H, W), dtype=torch.uint8, device="cuda")
    stats = []
    for i in range(NF2):
        stats.append(cog.cog_apply(ctx, te[i], m, want_stats=True))
        gm[i] = m.reshape(-1)[pt].cpu().numpy()
    gs_state = cog.decode_state(cog.cog_export_state(ctx, p), p)
    cog.cog_destroy(ctx)
    flags = [s["illum_flag"] for s in stats]
    assert flags[0] == 0
    assert flags[21] == 1 and sum(flags) <= 3, flags

    od = dict(d, width=len(pix), height=1)
    o = oracle.Oracle(od)
    trs = np.stack([sc.render(t, pix)[0] for t in range(NT)])
    ever = o.train(trs, want_near=True) != 0
    bad = agree = 0
    for i in range(NF2):
        o.state.illum[0] = len(pix) if flags[i] else 0   # this frame's flag
        f, _ = sc.render(NT + i, pix)
        om, _, near, st = o.apply(f)
        assert st["illum_flag"] == flags[i]
        ever |= near != 0
        bad += int(((gm[i] != om) & ~ever).sum())
        agree += int((gm[i] == om).sum())
    assert bad == 0
    assert agree / (NF2 * len(pix)) >= 0.9999
    ok = ~ever
    for k in ("w", "mu", "var", "rga_m", "rga_v", "conf"):
        e = rel_err(gs_state[k][pix][ok], getattr(o.state, k)[ok]).max()
        assert e <= 1e-4, (k, e)
