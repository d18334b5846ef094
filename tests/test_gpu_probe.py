"""The streaming probe that the benchmark times as the memory floor of a
stage-0-sized pass: it must do exactly the work its header defines (every
load feeds a store, so the timed pass moves all 16 bytes per pixel) and
write nothing outside its outputs."""
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


@pytest.mark.parametrize("P", [4, 516, 128 * 4 * 3 + 12, 1920 * 1080])
def test_probe_stream_output(cog, P):
    g = torch.Generator().manual_seed(P)
    dev = "cuda"
    jl = torch.randint(0, 2**31, (P,), generator=g, dtype=torch.int64).to(torch.int32).to(dev)
    conf = torch.randint(0, 2**15, (P,), generator=g, dtype=torch.int16).to(dev)
    frame = torch.randint(0, 256, (P, 3), generator=g, dtype=torch.uint8).to(dev)
    pad = 64   # canary elements after each output
    jl_o = torch.full((P + pad,), 0x5A5A5A5A, dtype=torch.int32, device=dev)
    conf_o = torch.full((P + pad,), 0x2B2B, dtype=torch.int16, device=dev)
    mask = torch.full((P + pad,), 0xC3, dtype=torch.uint8, device=dev)
    cog.cog_probe_stream(jl, conf, frame, jl_o[:P], conf_o[:P], mask[:P],
                         torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    f = frame.to(torch.int64)
    lab = (jl.to(torch.int64) & 0xFFFFFFFF) >> 24
    want = f[:, 0] | (f[:, 1] << 8) | (f[:, 2] << 16) | (lab << 24)
    assert torch.equal(jl_o[:P].to(torch.int64) & 0xFFFFFFFF, want)
    assert torch.equal(conf_o[:P], conf)
    assert torch.equal(mask[:P].to(torch.int64), lab)
    assert bool((jl_o[P:] == 0x5A5A5A5A).all())
    assert bool((conf_o[P:] == 0x2B2B).all())
    assert bool((mask[P:] == 0xC3).all())
