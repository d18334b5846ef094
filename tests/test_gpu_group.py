"""Spatio-temporal grouping (Sec. 2, "Clustering Similar Background -
Spatio-Temporal Grouping", steps 1-6 and Eq. 3) through the C ABI against
the FP64 oracle.

* Features: the GPU replays the warm-up in FP32, the oracle in FP64, so the
  codes agree within rounding except where a warm-up decision was near its
  threshold (the oracle's training near record): there a rank near-tie can
  change which mode is dominant for a frame.
* Clustering: the GPU evaluates the K-means distance in FP32, the oracle in
  FP64 with a near-tie record (the two nearest distances within 1e-5
  relative or within the bound on an FP32 evaluation's error).  The GPU's
  clustering is followed step by step (cog_group_cluster with a step
  limit), teacher-forced: from the GPU's labels after step s - 1 the
  oracle's Lloyd update and FP64 assignment must give the GPU's labels
  after step s on every pixel that is not near.  The Eq. 3 cores, counts
  and sums of the GPU's final labels must equal the oracle's for those
  labels exactly, and the iteration count must equal the teacher-forced
  one unless a near pixel went the other way.  With no near event along
  the way, the free-running FP64 clustering equals the GPU's outright.
* Step 6 reads the trained state, stored in the state dtype: its means agree
  within that dtype's rounding.
"""
import numpy as np
import pytest

from cog_harness import GpuRun, oracle_run, params

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

# step-6 tolerance: relative error of a core mean read from the stored state
PARAM_RTOL = {"f32": 1e-4, "f16": 2e-3, "bf16": 8e-3}


@pytest.fixture(scope="module")
def cog():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1705_09339_gb300 import cog
    return cog


def _frames(W, H, NT, kind, seed):
    from cogsynth import Scene
    sc = Scene(W, H, seed, kind=kind, n_train=NT, fg_frac=0.03)
    fr, _ = sc.frames(0, NT)
    return fr


def _gpu_group(d, dtype, fr):
    g = GpuRun(d, dtype)
    t = g._dev_frames(fr)
    g.cog.cog_train_prior(g.ctx, t, t.shape[0])
    P = d["width"] * d["height"]
    codes = torch.empty((2, P), dtype=torch.int16, device="cuda")
    labels = torch.empty(P, dtype=torch.uint8, device="cuda")
    st = g.cog.cog_group(g.ctx, t, t.shape[0], codes, labels)
    return g, st, codes.cpu().numpy().view(np.uint16), labels.cpu().numpy()


def _check_codes(gc, oc, near):
    """Within one code plus 1e-4 relative where no warm-up decision was near
    a threshold; returns the fraction of pixels that agree that closely."""
    ok = np.ones(gc.shape[1], bool)
    for f in range(2):
        a, b = gc[f].astype(np.int64), oc[f].astype(np.int64)
        ok &= np.abs(a - b) <= 1 + 1e-4 * np.maximum(a, b)
    clear = near == 0
    assert ok[clear].all(), (np.flatnonzero(~ok & clear)[:8], gc[:, ~ok & clear][:, :8], oc[:, ~ok & clear][:, :8])
    return ok.mean()


def _follow_steps(cog, ctx, gc, st_full):
    """Teacher-forced comparison of the GPU's clustering with the FP64
    oracle, step by step; returns the number of near pixels that went the
    other way on the GPU."""
    import oracle
    P = gc.shape[1]
    codes = torch.from_numpy(gc.view(np.int16).copy()).cuda()
    labels = torch.empty(P, dtype=torch.uint8, device="cuda")
    c, sd = oracle.group_init(gc[0], gc[1])
    prev, flips, s = None, 0, 0
    while True:
        st = cog.cog_group_cluster(ctx, codes, s, labels)
        gl = labels.cpu().numpy() & 0x7F
        if s > 0:
            c = oracle.group_centroids(gc[0], gc[1], prev, c)
        ol, near = oracle.group_assign(gc[0], gc[1], c, sd)
        bad = (gl != ol) & ~near
        assert not bad.any(), (s, np.flatnonzero(bad)[:8])
        flips += int(((gl != ol) & near).sum())
        if s > 0 and np.array_equal(gl, prev):
            break
        if s > 0:
            assert not st["converged"]
        prev, s = gl, s + 1
        assert s <= 64
    # the GPU's own run stops at the step that changed nothing
    assert st["converged"] == 1 and st["iterations"] == s
    assert st_full["converged"] == 1 and st_full["iterations"] == s
    return flips


def _check_cluster(cog, ctx, gc, gl, st):
    """The final labels, cores and sums against the oracle (see the module
    docstring); returns the free-running oracle's result."""
    import oracle
    flips = _follow_steps(cog, ctx, gc, st)
    cl, r = oracle.group_cores(gc[0], gc[1], gl & 0x7F)
    assert np.array_equal(gl, cl)                       # Eq. 3 cores of the GPU's clusters
    assert st["n"] == r["n"] and st["n_core"] == r["n_core"]
    assert st["code_sum"] == r["s1"] and st["code_sq_sum"] == r["s2"]
    for j in range(3):
        assert np.allclose(st["centroid"][j], r["centroid"][j], rtol=1e-12, atol=0)
        assert np.allclose(st["sd"][j], r["sd"][j], rtol=1e-12, atol=1e-12)
    ol, rf = oracle.group_cluster(gc[0], gc[1])
    if flips == 0 and rf["n_near"] == 0:
        assert np.array_equal(gl, ol) and rf["iterations"] == st["iterations"]
    else:
        assert (gl == ol).mean() >= 0.999
    return rf


def _check_params(st, o, gl, dtype):
    op = o.group_params(gl)
    tol = PARAM_RTOL[dtype]
    for j in range(3):
        if st["n_core"][j] == 0:
            continue
        assert st["w1"][j] == pytest.approx(op["w1"][j], rel=tol)
        assert st["mu1"][j] == pytest.approx(op["mu1"][j], rel=tol)
        assert st["v1"][j] == pytest.approx(op["v1"][j], rel=tol)


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("W,H,K,NT,kind", [(160, 120, 3, 200, "rects"), (96, 64, 5, 120, "dynamic")])
def test_group_matches_oracle(cog, dtype, W, H, K, NT, kind):
    fr = _frames(W, H, NT, kind, seed=3)
    d = params(W, H, K)
    g, st, gc, gl = _gpu_group(d, dtype, fr)
    o = oracle_run(d)
    near = o.train(fr, want_near=True)
    oc = np.stack(o.group_features(fr))
    frac = _check_codes(gc, oc, near)
    assert frac >= 0.995, frac
    r = _check_cluster(cog, g.ctx, gc, gl, st)
    g.close()
    assert r["converged"] == 1 and sum(st["n"]) == W * H
    assert (gl & 0x7F).max() <= 2
    _check_params(st, o, gl, dtype)


def test_group_is_deterministic(cog):
    fr = _frames(128, 72, 80, "dynamic", seed=5)
    d = params(128, 72, 3)
    g, st1, gc1, gl1 = _gpu_group(d, "f16", fr)
    t = g._dev_frames(fr)
    codes = torch.empty((2, 128 * 72), dtype=torch.int16, device="cuda")
    labels = torch.empty(128 * 72, dtype=torch.uint8, device="cuda")
    st2 = g.cog.cog_group(g.ctx, t, 80, codes, labels)
    g.close()
    assert np.array_equal(gc1, codes.cpu().numpy().view(np.uint16))
    assert np.array_equal(gl1, labels.cpu().numpy())
    for k in ("iterations", "converged", "n", "n_core", "code_sum", "code_sq_sum"):
        assert st1[k] == st2[k], k
    for j in range(3):
        assert st2["w1"][j] == pytest.approx(st1["w1"][j], rel=1e-12)


@pytest.mark.parametrize("W,H,K", [(1, 1, 1), (5, 3, 2), (33, 1, 8)])
def test_group_tiny_frames(cog, W, H, K):
    rng = np.random.default_rng(W * 100 + H)
    fr = rng.integers(0, 256, (12, W * H, 3), dtype=np.uint8)
    d = params(W, H, K)
    g, st, gc, gl = _gpu_group(d, "f32", fr)
    o = oracle_run(d)
    near = o.train(fr, want_near=True)
    _check_codes(gc, np.stack(o.group_features(fr)), near)
    _check_cluster(cog, g.ctx, gc, gl, st)
    g.close()


def test_group_cluster_hand_made_codes(cog):
    # three well separated groups of codes plus pixels on a tie between the
    # first two: clustering through cog_group_cluster alone (no features)
    rng = np.random.default_rng(11)
    W, H = 64, 40
    P = W * H
    centres = [(300, 200), (2600, 200), (900, 30000)]
    who = rng.integers(0, 3, P)
    v = np.array([centres[k][0] for k in who]) + rng.integers(-60, 61, P)
    w = np.array([centres[k][1] for k in who]) + rng.integers(-60, 61, P)
    gc = np.stack([v, w]).astype(np.uint16)
    d = params(W, H, 3)
    g = GpuRun(d, "f32")
    fr = torch.zeros((4, H, W, 3), dtype=torch.uint8, device="cuda")
    g.cog.cog_train_prior(g.ctx, fr, 4)
    codes = torch.from_numpy(gc.view(np.int16).copy()).cuda()
    labels = torch.empty(P, dtype=torch.uint8, device="cuda")
    st = cog.cog_group_cluster(g.ctx, codes, 64, labels)
    gl = labels.cpu().numpy()
    _check_cluster(cog, g.ctx, gc, gl, st)
    cl = gl & 3
    for k in range(3):
        assert len(set(cl[who == k])) == 1
    with pytest.raises(cog.CogError):
        cog.cog_group_cluster(g.ctx, codes, 65, labels)
    with pytest.raises(cog.CogError):
        cog.cog_group_cluster(g.ctx, codes, -1, labels)
    g.close()


def test_group_refuses_perchan_and_untrained(cog):
    d = params(16, 8, 3, flags=15 | 64)
    g = GpuRun(d, "f32")
    fr = torch.zeros((4, 8, 16, 3), dtype=torch.uint8, device="cuda")
    codes = torch.empty((2, 128), dtype=torch.int16, device="cuda")
    labels = torch.empty(128, dtype=torch.uint8, device="cuda")
    with pytest.raises(cog.CogError):
        cog.cog_group(g.ctx, fr, 4, codes, labels)     # before training
    g.cog.cog_train_prior(g.ctx, fr, 4)
    with pytest.raises(cog.CogError):
        cog.cog_group(g.ctx, fr, 4, codes, labels)     # per-channel mixtures
    g.close()


def test_group_full_size_1080p(cog):
    # the 1920x1080 dynamic-background stream with the bench's 500 training
    # frames: exact clustering of the whole frame given the GPU's codes;
    # features compared on 4096 sampled pixels (the warm-up is per pixel, so
    # the oracle runs on those pixels' time series alone)
    from cogsynth import workload
    from cogsynth.gpu import GpuScene
    sc = workload("hd_dynamic", fg_frac=0.02, seed=3)["scene"]
    train = GpuScene(sc, torch.device("cuda")).render(0, 500)
    d = params(1920, 1080, 5)
    g = GpuRun(d, "f16")
    g.cog.cog_train_prior(g.ctx, train, 500)
    P = 1920 * 1080
    codes = torch.empty((2, P), dtype=torch.int16, device="cuda")
    labels = torch.empty(P, dtype=torch.uint8, device="cuda")
    st = g.cog.cog_group(g.ctx, train, 500, codes, labels)
    gc = codes.cpu().numpy().view(np.uint16)
    gl = labels.cpu().numpy()
    r = _check_cluster(cog, g.ctx, gc, gl, st)
    g.close()
    assert r["converged"] == 1
    idx = np.random.default_rng(0).choice(P, 4096, replace=False)
    sub = train.reshape(500, P, 3)[:, torch.from_numpy(idx).cuda()].cpu().numpy()
    ds = params(4096, 1, 5)
    o = oracle_run(ds)
    near = o.train(sub, want_near=True)
    frac = _check_codes(gc[:, idx], np.stack(o.group_features(sub)), near)
    assert frac >= 0.995, frac
