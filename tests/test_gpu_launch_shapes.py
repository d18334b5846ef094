"""Launch shapes change speed, never results: every shape the autotuner
may pick gives bit-identical masks and model state; the tuner returns one
of its candidates and caches it."""
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


def test_every_launch_shape_gives_identical_results(cog):
    from cogsynth import Scene
    W, H, K, NT, NF = 333, 211, 5, 25, 6
    sc = Scene(W, H, 77, kind="dynamic", n_train=NT, fg_frac=0.08, switch_at=2)
    fr, _ = sc.frames(0, NT + NF)
    t = torch.from_numpy(fr.reshape(NT + NF, H, W, 3)).cuda()
    ref = None
    for shape in [(128, 64, 0), (64, 128, 0), (256, 64, 4), (128, 128, 1), (64, 64, 8)]:
        p = cog.cog_default_params(W, H, K, state_dtype="f16")
        c = cog.cog_create(p, torch.cuda.current_stream().cuda_stream)
        cog.cog_set_launch(c, *shape)
        cog.cog_train_prior(c, t[:NT], NT)
        m = torch.empty((NF, H, W), dtype=torch.uint8, device="cuda")
        for i in range(NF):
            cog.cog_apply(c, t[NT + i], m[i])
        st = cog.decode_state(cog.cog_export_state(c, p), p)
        out = (m.cpu().numpy(), st)
        cog.cog_destroy(c)
        if ref is None:
            ref = out
            continue
        assert np.array_equal(out[0], ref[0]), shape
        for k in ("w", "mu", "var", "rga_m", "rga_v", "conf", "label", "prev"):
            assert np.array_equal(out[1][k], ref[1][k]), (shape, k)


def test_bad_launch_shapes_rejected(cog):
    p = cog.cog_default_params(64, 64, 3)
    c = cog.cog_create(p, None)
    for bad in [(32, 64, 0), (128, 256, 0), (128, 64, -1)]:
        with pytest.raises(cog.CogError):
            cog.cog_set_launch(c, *bad)
    cog.cog_destroy(c)


def test_autotuner_picks_and_caches_a_candidate(cog, tmp_path):
    from cogsynth import Scene
    from paper_1705_09339_gb300 import autotune
    W, H, K = 320, 240, 3
    sc = Scene(W, H, 5, kind="dynamic", n_train=20, fg_frac=0.05)
    fr, _ = sc.frames(0, 30)
    t = torch.from_numpy(fr.reshape(30, H, W, 3)).cuda()
    p = cog.cog_default_params(W, H, K)
    cands = [(128, 64, 0), (256, 128, 0)]
    path = str(tmp_path / "cache.json")
    r = autotune.tune(p, t[:20], t[20:], n_frames=5, warmup=2, path=path, candidates=cands)
    assert tuple(r["best"]) in cands and len(r["us"]) == 2
    c = cog.cog_create(p, None)
    assert autotune.apply_best(c, p, path) == tuple(r["best"])
    cog.cog_destroy(c)
