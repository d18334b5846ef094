"""The clip path (cog_apply_clip: up to 32 frames per cooperative launch,
stage-0/1 state on chip across them) against frame-by-frame cog_apply.

The two compute the same per-pixel steps with the same arithmetic and the
same rounding to the storage type after every frame, so masks, stage maps,
per-frame counts, illumination flags and the final state must be
bit-identical for every storage type -- including clips whose speculated
illumination flags are wrong (a light switch inside the clip), which the
kernel detects and reruns.  The clip path is also checked against the FP64
oracle like the per-frame path.
"""
import numpy as np
import pytest

from cog_harness import GpuRun, compare_stream, oracle_run, params, state_errors, oracle_state

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _pair(d, dtype, train):
    a, b = GpuRun(d, dtype), GpuRun(d, dtype)
    a.train(train)
    b.train(train)
    return a, b


def _clip(g, frames, chunks):
    """Applies frames [n, H, W, 3] (device) as clips of the given sizes."""
    cog, torch_ = g.cog, g.torch
    n = frames.shape[0]
    masks = torch_.empty((n, g.P), dtype=torch_.uint8, device="cuda")
    stages = torch_.empty((n, g.P), dtype=torch_.uint8, device="cuda")
    st, i = [], 0
    for c in chunks:
        st += cog.cog_apply_clip(g.ctx, frames[i:i + c], c, masks[i:i + c], stages[i:i + c], want_stats=True)
        i += c
    assert i == n
    cog.cog_sync(g.ctx)
    return masks.cpu().numpy(), stages.cpu().numpy(), st


def _same_state(a, b):
    sa, sb = a.state(), b.state()
    for k in sa:
        assert np.array_equal(sa[k], sb[k]), k


def _scene(W, H, seed, NT, NF, **kw):
    from cogsynth import Scene
    from cogsynth.gpu import GpuScene
    sc = Scene(W, H, seed, n_train=NT, **kw)
    return GpuScene(sc).render(0, NT + NF)


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("K", [3, 5])
def test_clip_equals_frame_by_frame(dtype, K):
    W, H, NT, NF = 320, 240, 60, 70
    fr = _scene(W, H, 4, NT, NF, kind="dynamic", fg_frac=0.05, switch_at=10 ** 6)
    d = params(W, H, K)
    a, b = _pair(d, dtype, fr[:NT])
    am, asg, ast = a.apply(fr[NT:])
    bm, bsg, bst = _clip(b, fr[NT:], [32, 32, 6])
    assert np.array_equal(am, bm)
    assert np.array_equal(asg, bsg)
    for t in range(NF):
        assert ast[t]["n_stage"] == bst[t]["n_stage"], t
        assert ast[t]["n_gmm"] == bst[t]["n_gmm"] and ast[t]["illum_flag"] == bst[t]["illum_flag"], t
    _same_state(a, b)
    # running totals and the next frame's counters continue identically
    assert a.cog.cog_read_stats(a.ctx) == b.cog.cog_read_stats(b.ctx)
    am, asg, _ = a.apply(fr[NT:NT + 3])
    bm, bsg, _ = b.apply(fr[NT:NT + 3])
    assert np.array_equal(am, bm) and np.array_equal(asg, bsg)
    a.close(); b.close()


@pytest.mark.parametrize("switch_at", [0, 5, 31])
def test_clip_with_light_switch_reruns_and_matches(switch_at):
    # the +60 switch makes frame s+1 (and often s+2) flagged: the clip's
    # speculation fails, it restores its state and runs again
    W, H, K, NT, NF = 160, 120, 3, 40, 40
    fr = _scene(W, H, 8, NT, NF, kind="dynamic", fg_frac=0.05, switch_at=switch_at)
    d = params(W, H, K)
    a, b = _pair(d, "f16", fr[:NT])
    am, asg, ast = a.apply(fr[NT:])
    bm, bsg, bst = _clip(b, fr[NT:], [32, 8])
    flags = [s["illum_flag"] for s in ast]
    assert sum(flags) >= 1
    assert flags == [s["illum_flag"] for s in bst]
    assert np.array_equal(am, bm) and np.array_equal(asg, bsg)
    _same_state(a, b)
    a.close(); b.close()


def test_clip_rerun_count():
    # no switch: one run; a switch inside the first launch: more than one
    W, H, K = 96, 64, 3
    for switch_at, expect_more in ((10 ** 6, False), (10, True)):
        fr = _scene(W, H, 3, 30, 32, kind="dynamic", fg_frac=0.05, switch_at=switch_at)
        g = GpuRun(params(W, H, K), "f32")
        g.train(fr[:30])
        _clip(g, fr[30:], [32])
        runs = g.cog.cog_clip_runs(g.ctx)
        g.close()
        assert (runs > 1) == expect_more, (switch_at, runs)


@pytest.mark.parametrize("W,H", [(37, 29), (1, 1), (1025, 3), (257, 2)])
def test_clip_ragged_sizes_and_unaligned_buffers(W, H):
    NT, NF = 20, 35
    fr = _scene(W, H, 6, NT, NF, kind="dynamic", fg_frac=0.1, switch_at=12)
    d = params(W, H, 3)
    a, b = _pair(d, "f32", fr[:NT])
    am, asg, _ = a.apply(fr[NT:])
    # frames and masks at odd byte offsets
    P = W * H
    fb = torch.zeros(NF * P * 3 + 1, dtype=torch.uint8, device="cuda")
    fb[1:].copy_(fr[NT:].reshape(-1))
    mb = torch.zeros(NF * P + 3, dtype=torch.uint8, device="cuda")
    sb = torch.zeros(NF * P + 1, dtype=torch.uint8, device="cuda")
    b.cog.cog_apply_clip(b.ctx, fb[1:], NF, mb[3:], sb[1:])
    b.cog.cog_sync(b.ctx)
    assert np.array_equal(am.reshape(-1), mb[3:].cpu().numpy())
    assert np.array_equal(asg.reshape(-1), sb[1:].cpu().numpy())
    _same_state(a, b)
    a.close(); b.close()


def test_clip_with_temporal_sampling_matches_frame_by_frame():
    W, H, K, NT, NF = 256, 96, 3, 40, 64
    fr = _scene(W, H, 9, NT, NF, kind="dynamic", fg_frac=0.03, switch_at=10 ** 6)
    d = params(W, H, K, flags=15 | 16)
    a, b = _pair(d, "f16", fr[:NT])
    am, asg, ast = a.apply(fr[NT:])
    bm, bsg, bst = _clip(b, fr[NT:], [7, 32, 25])
    assert sum(s["n_stage"][5] for s in ast) > 0
    assert np.array_equal(am, bm) and np.array_equal(asg, bsg)
    assert [s["n_stage"] for s in ast] == [s["n_stage"] for s in bst]
    _same_state(a, b)
    a.close(); b.close()


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_clip_mode1_equals_frame_by_frame(dtype):
    W, H, K, NT, NF = 200, 150, 5, 40, 50
    fr = _scene(W, H, 5, NT, NF, kind="dynamic", fg_frac=0.05, switch_at=30)
    d = params(W, H, K, flags=15 | 32)
    a, b = _pair(d, dtype, fr[:NT])
    am, asg, ast = a.apply(fr[NT:])
    bm, bsg, bst = _clip(b, fr[NT:], [32, 18])
    assert np.array_equal(am, bm) and np.array_equal(asg, bsg)
    assert [s["illum_flag"] for s in ast] == [s["illum_flag"] for s in bst]
    _same_state(a, b)
    a.close(); b.close()


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_clip_perchan_equals_frame_by_frame(dtype):
    W, H, K, NT, NF = 200, 150, 5, 40, 50
    fr = _scene(W, H, 12, NT, NF, kind="dynamic", fg_frac=0.05, switch_at=30)
    d = params(W, H, K, flags=15 | 64)
    a, b = _pair(d, dtype, fr[:NT])
    am, asg, ast = a.apply(fr[NT:])
    bm, bsg, bst = _clip(b, fr[NT:], [32, 18])
    assert np.array_equal(am, bm) and np.array_equal(asg, bsg)
    assert [s["illum_flag"] for s in ast] == [s["illum_flag"] for s in bst]
    _same_state(a, b)
    a.close(); b.close()


def test_clip_fp32_matches_oracle():
    # the 160x120 workload through the clip path against the FP64 oracle
    from cogsynth import Scene
    W, H, K, NT, NF = 160, 120, 3, 200, 300
    sc = Scene(W, H, 1, kind="rects", n_train=NT, fg_frac=0.03)
    fr, _ = sc.frames(0, NT + NF)
    d = params(W, H, K)
    g = GpuRun(d, "f32")
    g.train(fr[:NT])
    gm, gsm, _ = _clip(g, torch.from_numpy(np.ascontiguousarray(fr[NT:])).cuda().reshape(NF, H, W, 3),
                       [32] * 9 + [12])
    gs = g.state()
    g.close()
    o = oracle_run(d)
    near0 = o.train(fr[:NT], want_near=True)
    om, osm, near = [], [], []
    for t in range(NF):
        m, s, n, _ = o.apply(fr[NT + t])
        om.append(m); osm.append(s); near.append(n)
    near[0] = near[0] | near0
    agree, unexplained, ever = compare_stream(gm, gsm, np.stack(om), np.stack(osm), np.stack(near))
    assert unexplained == 0 and agree >= 0.9999
    e = state_errors(gs, oracle_state(o), ~ever)
    for k in ("w", "mu", "var", "rga_m", "rga_v", "conf"):
        assert e[k] <= TOL, (k, e[k])


def test_clip_and_frames_interleave():
    # per-frame, clip, per-frame, clip on one context == all per-frame
    W, H, K, NT = 128, 80, 5, 30
    fr = _scene(W, H, 2, NT, 50, kind="dynamic", fg_frac=0.05, switch_at=23)
    d = params(W, H, K)
    a, b = _pair(d, "bf16", fr[:NT])
    am, asg, _ = a.apply(fr[NT:])
    parts_m, parts_s = [], []
    m, s, _ = b.apply(fr[NT:NT + 3]); parts_m.append(m); parts_s.append(s)
    m, s, _ = _clip(b, fr[NT + 3:NT + 20], [17]); parts_m.append(m); parts_s.append(s)
    m, s, _ = b.apply(fr[NT + 20:NT + 21]); parts_m.append(m); parts_s.append(s)
    m, s, _ = _clip(b, fr[NT + 21:NT + 50], [29]); parts_m.append(m); parts_s.append(s)
    assert np.array_equal(am, np.concatenate(parts_m)) and np.array_equal(asg, np.concatenate(parts_s))
    _same_state(a, b)
    assert a.cog.cog_read_stats(a.ctx) == b.cog.cog_read_stats(b.ctx)
    a.close(); b.close()
