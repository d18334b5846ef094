"""The batched path (many streams per step in one captured graph) gives
exactly what per-stream cog_apply gives, through graph replays, mixed
sizes, K and storage types, and changing frame buffers."""
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


# "+pc": per-channel mixtures, "+m1": stage 1 as the rank-1 mode (each a
# group of its own in the batch); "+q4": the 4-bit scene prior (in the same
# group as the 8-bit streams)
SPECS = [(160, 120, 3, "f32"), (320, 240, 5, "f16"), (97, 61, 3, "f32"), (640, 480, 5, "f16"),
         (33, 1, 5, "f16"), (200, 100, 3, "bf16"), (160, 120, 5, "f16"), (128, 96, 5, "f16+pc"),
         (64, 48, 3, "f32+pc"), (176, 144, 5, "f16+q4"), (45, 31, 3, "f32+pc+q4"), (120, 90, 5, "f16+m1"),
         (96, 40, 3, "f32+m1+q4")]


def _streams(n_train=20, n_test=6):
    from cogsynth import Scene
    out = []
    for i, (w, h, k, dt) in enumerate(SPECS):
        sc = Scene(w, h, 40 + i, kind="dynamic", n_train=n_train, fg_frac=0.05, switch_at=3)
        fr, _ = sc.frames(0, n_train + n_test)
        out.append((w, h, k, dt, fr))
    return out


def _ctx(cog, w, h, k, dt, fr, n_train, stream):
    base, *opts = dt.split("+")
    p = cog.cog_default_params(w, h, k, state_dtype=base)
    if "pc" in opts:
        p.flags |= cog.COG_PERCHAN
    if "q4" in opts:
        p.kde_bits = 4
    if "m1" in opts:
        p.flags |= cog.COG_MODE1
    c = cog.cog_create(p, stream)
    t = torch.from_numpy(fr[:n_train].reshape(n_train, h, w, 3)).cuda()
    cog.cog_train_prior(c, t, n_train)
    cog.cog_sync(c)
    return c, p


def test_batch_equals_single_stream_apply(cog):
    NT, NF = 20, 6
    data = _streams(NT, NF)
    s = torch.cuda.Stream()
    single = [_ctx(cog, w, h, k, dt, fr, NT, s.cuda_stream) for (w, h, k, dt, fr) in data]
    batched = [_ctx(cog, w, h, k, dt, fr, NT, s.cuda_stream) for (w, h, k, dt, fr) in data]
    b = cog.cog_batch_create([c for c, _ in batched], s.cuda_stream)
    # two sets of device frame buffers, alternated between steps
    bufs = [[torch.empty((h, w, 3), dtype=torch.uint8, device="cuda") for (w, h, _, _, _) in data] for _ in range(2)]
    mb = [torch.empty((h, w), dtype=torch.uint8, device="cuda") for (w, h, _, _, _) in data]
    ms = [torch.empty((h, w), dtype=torch.uint8, device="cuda") for (w, h, _, _, _) in data]
    for t in range(NF):
        with torch.cuda.stream(s):
            for i, (w, h, k, dt, fr) in enumerate(data):
                bufs[t % 2][i].copy_(torch.from_numpy(fr[NT + t].reshape(h, w, 3)))
            s.synchronize()
            for i, (c, _) in enumerate(single):
                cog.cog_apply(c, bufs[t % 2][i], ms[i])
            cog.cog_batch_apply(b, bufs[t % 2], mb)
            cog.cog_batch_sync(b)
            for c, _ in single:
                cog.cog_sync(c)
        for i in range(len(data)):
            assert torch.equal(mb[i], ms[i]), (t, i)
    for (ca, pa), (cb, pb) in zip(single, batched):
        sa = cog.decode_state(cog.cog_export_state(ca, pa), pa)
        sb = cog.decode_state(cog.cog_export_state(cb, pb), pb)
        for key in ("w", "wc", "mu", "var", "rga_m", "rga_v", "conf", "label", "prev"):
            if key in sa:
                assert np.array_equal(sa[key], sb[key]), key
        la, ta = cog.cog_read_stats(ca)
        lb, tb = cog.cog_read_stats(cb)
        assert la == lb and ta == tb
    cog.cog_batch_destroy(b)
    for c, _ in single + batched:
        cog.cog_destroy(c)


def test_batch_argument_errors(cog):
    with pytest.raises(cog.CogError):
        cog.cog_batch_create([], torch.cuda.Stream().cuda_stream)
    p = cog.cog_default_params(32, 32, 3)
    c = cog.cog_create(p, None)
    with pytest.raises(cog.CogError) as e:          # untrained
        cog.cog_batch_create([c], torch.cuda.Stream().cuda_stream)
    assert e.value.status == cog.COG_ERR_STATE
    cog.cog_destroy(c)


def test_batch_matches_oracle_with_inactive_steps(cog):
    # four small streams of mixed size, K = 3 and 5, FP32 state, through
    # cog_batch_apply_active with each stream idle on some steps; every
    # stream is compared with its own FP64 oracle run over the frames it
    # actually received: masks identical on every pixel with no decision
    # near a threshold so far, state within 1e-4 relative there; two of the
    # streams keep the 4-bit prior
    specs = [(97, 61, 3, 8), (160, 120, 5, 4), (33, 7, 5, 8), (200, 100, 3, 4)]
    NT, NF = 40, 30
    s = torch.cuda.Stream()      # a graph cannot be captured on the legacy default stream
    with torch.cuda.stream(s):
        _batch_vs_oracle(cog, specs, NT, NF, s)


def _batch_vs_oracle(cog, specs, NT, NF, s):
    from cog_harness import GpuRun, oracle_run, oracle_state, params, state_errors
    from cogsynth import Scene
    runs = []
    for i, (w, h, k, bits) in enumerate(specs):
        sc = Scene(w, h, 90 + i, kind="dynamic", n_train=NT, fg_frac=0.05, switch_at=12 + 3 * i)
        fr, _ = sc.frames(0, NT + NF)
        d = params(w, h, k, kde_bits=bits)
        g = GpuRun(d, "f32")
        g.train(fr[:NT])
        runs.append((w, h, k, fr, d, g))
    b = cog.cog_batch_create([r[5].ctx for r in runs], s.cuda_stream)
    used = [0] * len(specs)
    got = [[] for _ in specs]
    for t in range(NF):
        active = [int((t + i) % 4 != 3 or t < 2) for i in range(len(specs))]
        frames, masks = [], []
        for i, (w, h, k, fr, d, g) in enumerate(runs):
            if active[i]:
                frames.append(torch.from_numpy(fr[NT + used[i]].reshape(h, w, 3)).cuda())
                masks.append(torch.empty((h, w), dtype=torch.uint8, device="cuda"))
            else:
                frames.append(None)
                masks.append(None)
        cog.cog_batch_apply_active(b, frames, masks, active)
        cog.cog_batch_sync(b)
        for i in range(len(specs)):
            if active[i]:
                got[i].append(masks[i].cpu().numpy().ravel())
                used[i] += 1
    cog.cog_batch_destroy(b)
    for i, (w, h, k, fr, d, g) in enumerate(runs):
        assert 0 < used[i] < NF
        gs = g.state()
        g.close()
        o = oracle_run(d)
        near0 = o.train(fr[:NT], want_near=True)
        ever = near0 != 0
        unexplained = 0
        for j in range(used[i]):
            m, _, near, _ = o.apply(fr[NT + j])
            ever |= near != 0
            unexplained += int(((got[i][j] != m) & ~ever).sum())
        assert unexplained == 0, (i, unexplained)
        e = state_errors(gs, oracle_state(o), ~ever)
        for key in ("w", "mu", "var", "rga_m", "rga_v", "conf"):
            assert e[key] <= 1e-4, (i, key, e[key])
        for key in ("label", "prev", "qa", "qb"):
            assert e[key] == 0, (i, key)


@pytest.mark.parametrize("K,dt,flags", [(5, "f16", 15), (3, "f32", 15 | 32), (5, "bf16", 15 | 64)])
def test_batch_many_survivors_per_thread(cog, K, dt, flags):
    # seeded random states and frames send most pixels to the mixture stage,
    # so each of the batch's mixture-stage threads walks many survivors (its
    # software pipeline runs many rounds); batched and single-stream
    # application must agree bit for bit
    from cog_harness import random_frame, random_state, to_cog, params
    W, H = 1280, 720
    P = W * H
    rng = np.random.default_rng(60 + K + flags)
    st = random_state(rng, P, K, dtype=dt, mode1=bool(flags & 32), perchan=bool(flags & 64), kde_const=60)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctxs = []
        for _ in range(2):
            p = to_cog(params(W, H, K, flags=flags), dt)
            c = cog.cog_create(p, s.cuda_stream)
            z = torch.zeros((2, H, W, 3), dtype=torch.uint8, device="cuda")
            cog.cog_train_prior(c, z, 2)
            buf = cog.cog_export_state(c, p)
            cog.cog_import_state(c, cog.encode_state(buf, p, st))
            ctxs.append((c, p))
        b = cog.cog_batch_create([ctxs[1][0]], s.cuda_stream)
        ms = torch.empty((H, W), dtype=torch.uint8, device="cuda")
        mb = torch.empty((H, W), dtype=torch.uint8, device="cuda")
        for t in range(3):
            f = torch.from_numpy(random_frame(rng, st, mix=(0.1, 0.5, 0.4)).reshape(H, W, 3)).cuda()
            cog.cog_apply(ctxs[0][0], f, ms)
            cog.cog_batch_apply(b, [f], [mb])
            cog.cog_batch_sync(b)
            cog.cog_sync(ctxs[0][0])
            assert torch.equal(ms, mb), t
        la, _ = cog.cog_read_stats(ctxs[0][0])
        lb, _ = cog.cog_read_stats(ctxs[1][0])
        assert la == lb and la["n_gmm"] > P // 3
        sa = cog.decode_state(cog.cog_export_state(*ctxs[0]), ctxs[0][1])
        sb = cog.decode_state(cog.cog_export_state(*ctxs[1]), ctxs[1][1])
        for key in ("w", "wc", "mu", "var", "rga_m", "rga_v", "conf", "label", "prev", "top"):
            if key in sa:
                assert np.array_equal(sa[key], sb[key]), key
        cog.cog_batch_destroy(b)
        for c, _ in ctxs:
            cog.cog_destroy(c)
