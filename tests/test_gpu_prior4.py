"""The 4-bit scene prior (kde_bits = 4) on the CUDA path against the FP64
oracle, through the C ABI.

Training is integer work and must be bit-exact: the GPU's nibble-packed
rows, unpacked, equal the oracle's levels of 15 at every size, bandwidth
and for the packing's odd and even grey levels.  Applying frames with the
4-bit prior follows the same bars as the 8-bit stream tests (masks and
stage maps identical away from the oracle's near record, state within
1e-4 relative); the clip path equals frame-by-frame application bit for bit.
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


@pytest.mark.parametrize("W,H,N,bw", [(37, 29, 23, 4), (1, 1, 2, 4), (160, 120, 200, 4), (53, 7, 31, 1),
                                      (45, 13, 19, 7)])
def test_prior4_training_bit_exact(W, H, N, bw):
    from cogsynth import Scene
    sc = Scene(W, H, 11, kind="dynamic", n_train=N, fg_frac=0.05)
    fr, _ = sc.frames(0, N)
    d = params(W, H, 3, kde_bw=bw, kde_bits=4)
    g = GpuRun(d)
    g.train(fr)
    gs = g.state()
    g.close()
    o = oracle_run(d)
    o.train(fr)
    os_ = oracle_state(o)
    assert gs["kde"].max() <= 15 and os_["kde"].max() == 15
    assert np.array_equal(gs["kde"], os_["kde"])
    assert np.array_equal(gs["qa"], os_["qa"]) and np.array_equal(gs["qb"], os_["qb"])


def test_prior4_halves_the_prior_plane():
    from paper_1705_09339_gb300 import cog
    p8 = cog.cog_default_params(1920, 1080, 5, state_dtype="f16")
    p4 = cog.cog_default_params(1920, 1080, 5, state_dtype="f16", kde_bits=4)
    L8, L4 = cog.cog_state_layout(p8), cog.cog_state_layout(p4)
    P = 1920 * 1080
    assert L8.total - L4.total >= P * 384 - 256
    assert L4.kde_row == 128


def test_prior4_stream_fp32_matches_oracle():
    # the 160x120 workload with the 4-bit prior: 200 training frames, 150
    # test frames, K = 3, FP32 state
    from cogsynth import Scene
    W, H, K, NT, NF = 160, 120, 3, 200, 150
    sc = Scene(W, H, 1, kind="rects", n_train=NT, fg_frac=0.03)
    fr, _ = sc.frames(0, NT + NF)
    d = params(W, H, K, kde_bits=4)
    g = GpuRun(d)
    g.train(fr[:NT])
    gm, gsm, gst = g.apply(fr[NT:])
    gs = g.state()
    g.close()
    o = oracle_run(d)
    near0 = o.train(fr[:NT], want_near=True)
    om, osm, near, ost = [], [], [], []
    for t in range(NF):
        m, s, n, st = o.apply(fr[NT + t])
        om.append(m); osm.append(s); near.append(n); ost.append(st)
    near[0] = near[0] | near0
    agree, unexplained, ever = compare_stream(gm, gsm, np.stack(om), np.stack(osm), np.stack(near))
    assert unexplained == 0
    assert agree >= 0.9999
    e = state_errors(gs, oracle_state(o), ~ever)
    for k in ("w", "mu", "var", "rga_m", "rga_v", "conf"):
        assert e[k] <= TOL, (k, e[k])
    for k in ("label", "prev", "qa", "qb"):
        assert e[k] == 0, k
    assert np.array_equal(gs["kde"], oracle_state(o)["kde"])


@pytest.mark.parametrize("K,flags", [(3, 15), (5, 15), (5, 15 | 64), (3, 15 | 32), (5, 4 | 8)])
def test_prior4_seeded_state_steps_match_oracle(K, flags):
    # random 4-bit levels (30 % at the nullified level 0) at every grey
    # level, so both nibbles of the packed rows are read
    rng = np.random.default_rng(400 + K * 16 + flags)
    W, H = 61, 37
    P = W * H
    d = params(W, H, K, flags=flags, kde_bits=4)
    st = random_state(rng, P, K, mode1=bool(flags & 32), perchan=bool(flags & 64), kde_bits=4)
    g = GpuRun(d)
    g.train(np.zeros((2, P, 3), np.uint8))
    g.set_state(st)
    assert np.array_equal(g.state()["kde"], st["kde"])
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
    e = state_errors(g.state(), oracle_state(o), ~ever)
    g.close()
    for k in ("w", "mu", "var", "rga_m", "rga_v", "conf", "wc"):
        if k in e:
            assert e[k] <= TOL, (k, e[k])


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_prior4_clip_equals_frame_by_frame(dtype):
    from cogsynth import Scene
    from cogsynth.gpu import GpuScene
    W, H, K, NT, NF = 200, 120, 5, 40, 40
    fr = GpuScene(Scene(W, H, 6, n_train=NT, kind="dynamic", fg_frac=0.05, switch_at=10 ** 6)).render(0, NT + NF)
    d = params(W, H, K, kde_bits=4)
    a, b = GpuRun(d, dtype), GpuRun(d, dtype)
    a.train(fr[:NT])
    b.train(fr[:NT])
    am, asg, ast = a.apply(fr[NT:])
    cog = b.cog
    masks = torch.empty((NF, b.P), dtype=torch.uint8, device="cuda")
    stages = torch.empty((NF, b.P), dtype=torch.uint8, device="cuda")
    bst = []
    for i in range(0, NF, 20):
        bst += cog.cog_apply_clip(b.ctx, fr[NT + i:NT + i + 20], 20, masks[i:i + 20], stages[i:i + 20],
                                  want_stats=True)
    cog.cog_sync(b.ctx)
    assert np.array_equal(am, masks.cpu().numpy()) and np.array_equal(asg, stages.cpu().numpy())
    assert [s["n_stage"] for s in ast] == [s["n_stage"] for s in bst]
    sa, sb = a.state(), b.state()
    for k in sa:
        assert np.array_equal(sa[k], sb[k]), k
    a.close(); b.close()
