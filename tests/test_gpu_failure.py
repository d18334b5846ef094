"""Failure detection and memory-safety checks that fault no GPU.

* The bounded grid-wide wait (the clip kernel's barrier) runs on a count
  that nothing completes: it must give up after its limit, set the error
  bit, and leave the device usable.
* Canary bytes around a caller-owned state buffer and around the output
  buffers must be untouched by training, per-frame and clip application,
  the plain mixture and state import/export.
"""
import numpy as np
import pytest

from cog_harness import GpuRun, params, to_cog

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

DERR_GRID_TIMEOUT = 2


@pytest.fixture(scope="module")
def cog():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1705_09339_gb300 import cog
    return cog


@pytest.mark.parametrize("limit_ms", [20, 200])
def test_bounded_wait_gives_up_and_reports(cog, limit_ms):
    err, ms = cog.cog_selftest_bounded_wait(limit_ms)
    assert err == DERR_GRID_TIMEOUT
    assert limit_ms * 0.9 <= ms <= limit_ms + 250, ms
    # the device is still usable afterwards
    d = params(64, 48, 3)
    g = GpuRun(d)
    g.train(np.random.default_rng(0).integers(0, 256, (4, 64 * 48, 3), dtype=np.uint8))
    m, _, _ = g.apply(np.zeros((2, 64 * 48, 3), np.uint8))
    g.close()
    assert m.shape == (2, 64 * 48)


def test_canaries_around_state_and_outputs(cog):
    from cogsynth import Scene
    W, H, K, NT, NF = 203, 77, 5, 30, 40        # ragged size
    P = W * H
    GUARD = 4096
    d = params(W, H, K, flags=15 | 16)
    p = to_cog(d, "f16")
    nbytes = cog.cog_state_bytes(p)
    buf = torch.full((nbytes + 2 * GUARD,), 0xA5, dtype=torch.uint8, device="cuda")
    ctx = cog.cog_create(p, torch.cuda.current_stream().cuda_stream, buf[GUARD:])
    sc = Scene(W, H, 4, kind="dynamic", n_train=NT, fg_frac=0.1, switch_at=15)
    fr, _ = sc.frames(0, NT + NF)
    fr = torch.from_numpy(np.ascontiguousarray(fr)).cuda().reshape(NT + NF, H, W, 3)
    cog.cog_train_prior(ctx, fr[:NT], NT)
    out = torch.full((3 * NF * P + 2 * GUARD,), 0x5A, dtype=torch.uint8, device="cuda")
    masks = out[GUARD:GUARD + NF * P].view(NF, P)
    smaps = out[GUARD + NF * P:GUARD + 2 * NF * P].view(NF, P)
    pmask = out[GUARD + 2 * NF * P:GUARD + 3 * NF * P].view(NF, P)
    for i in range(NF // 2):
        cog.cog_apply(ctx, fr[NT + i], masks[i], smaps[i])
    cog.cog_apply_clip(ctx, fr[NT + NF // 2:], NF - NF // 2, masks[NF // 2:], smaps[NF // 2:])
    for i in range(NF):
        cog.cog_apply_plain_gmm(ctx, fr[NT + i], pmask[i])
    img = cog.cog_export_state(ctx, p)
    cog.cog_import_state(ctx, img)
    cog.cog_sync(ctx)
    cog.cog_destroy(ctx)
    torch.cuda.synchronize()
    assert bool((buf[:GUARD] == 0xA5).all()) and bool((buf[GUARD + nbytes:] == 0xA5).all())
    assert bool((out[:GUARD] == 0x5A).all()) and bool((out[GUARD + 3 * NF * P:] == 0x5A).all())
