"""Accuracy per configuration against the FP64 oracle and the ground truth.

For the 160x120 workload (K=3, 200 training + 300 test frames) and the
640x480 dynamic workload (K=5, 500 training + 1000 test frames, with the +60
light switch at test frame 600), the CUDA path runs with FP32, FP16 and BF16
model state; the oracle runs once.  Reported (and written to
accuracy_report.json in the run's output folder): mask agreement with the oracle, mismatches
not explained by near-threshold decisions, relative error of the final means
and variances, and the misclassification rate against the generator's
ground truth for the cascade (GPU) and the plain mixture (GPU, same frames).
FP32 must match the oracle (>= 99.99 %, no unexplained mismatch); 16-bit
storage agreement is stated, with floors FP16 >= 99 % and BF16 >= 95 %.
On the dynamic-background workload (blobs, sway, light switch) the cascade
must misclassify fewer pixels than the plain mixture; on the 160x120
workload, whose slow +20 brightness ramp leaves the models of pixels that
exit early stale, the cascade's higher error is reported, not asserted.
"""
import json
import os

import numpy as np
import pytest

from cog_harness import GpuRun, compare_stream, oracle_run, params, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

CONFIGS = {
    "qvga_rects": dict(W=160, H=120, K=3, NT=200, NF=300, kind="rects", seed=1, fg=0.03, switch=10 ** 6),
    "vga_dynamic": dict(W=640, H=480, K=5, NT=500, NF=1000, kind="dynamic", seed=2, fg=0.03, switch=600),
}
FLOORS = {"f32": 0.9999, "f16": 0.99, "bf16": 0.95}
REPORT = {}


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    yield
    # the per-config report goes where COG_REPORT_DIR points (nowhere if unset)
    out = os.environ.get("COG_REPORT_DIR")
    if out:
        os.makedirs(out, exist_ok=True)
        with open(os.path.join(out, "accuracy_report.json"), "w") as f:
            json.dump(REPORT, f, indent=1)


def _misclass(masks, gt):
    return float(((masks > 0) != (gt > 0)).mean())


@pytest.mark.parametrize("name", list(CONFIGS))
def test_accuracy_per_config(name):
    from cogsynth import Scene
    from cogsynth.gpu import GpuScene
    c = CONFIGS[name]
    W, H, K, NT, NF = c["W"], c["H"], c["K"], c["NT"], c["NF"]
    sc = Scene(W, H, c["seed"], kind=c["kind"], n_train=NT, fg_frac=c["fg"], switch_at=c["switch"])
    gs = GpuScene(sc)
    frames_d, gt_d = gs.render(0, NT + NF, gt=True)
    frames = frames_d.cpu().numpy().reshape(NT + NF, -1, 3)
    gt = gt_d.cpu().numpy().reshape(NT + NF, -1)[NT:]
    d = params(W, H, K)
    o = oracle_run(d)
    near0 = o.train(frames[:NT], want_near=True)
    om, osm, near = [], [], []
    for t in range(NF):
        m, s, n, _ = o.apply(frames[NT + t])
        om.append(m); osm.append(s); near.append(n)
    near[0] = near[0] | near0   # warm-up decisions near a threshold count too
    om, osm, near = np.stack(om), np.stack(osm), np.stack(near)
    rep = {"pixels": W * H, "test_frames": NF, "oracle_misclass_vs_truth": _misclass(om, gt)}
    for dtype in ("f32", "f16", "bf16"):
        g = GpuRun(d, dtype)
        g.train(frames_d[:NT])
        gm, gsm, _ = g.apply(frames_d[NT:], stats=False)
        st = g.state()
        g.close()
        agree, unexplained, ever = compare_stream(gm, gsm, om, osm, near)
        ok = ~ever
        errs = {k: float(np.percentile(rel_err(st[k][ok], getattr(o.state, k)[ok]), 99)) if ok.any() else 0.0
                for k in ("w", "mu", "var")}
        rep[dtype] = {"mask_agreement": agree, "unexplained_mismatches": unexplained,
                      "p99_rel_err_final_state": errs, "misclass_vs_truth": _misclass(gm, gt)}
        assert agree >= FLOORS[dtype], (name, dtype, agree)
        if dtype == "f32":
            assert unexplained == 0
    p = GpuRun(params(W, H, K, flags=0), "f16")
    p.train(frames_d[:NT])
    pm, _, _ = p.apply(frames_d[NT:], stats=False, plain=True)
    p.close()
    rep["plain_gmm_f16_misclass_vs_truth"] = _misclass(pm, gt)
    # the Fig. 1 reading (COG_MODE1): oracle and FP16 GPU, reported
    o1 = oracle_run(params(W, H, K, flags=15 | 32))
    o1.train(frames[:NT])
    m1 = np.stack([o1.apply(frames[NT + t], want_stage=False, want_near=False)[0] for t in range(NF)])
    g1 = GpuRun(params(W, H, K, flags=15 | 32), "f16")
    g1.train(frames_d[:NT])
    gm1, _, _ = g1.apply(frames_d[NT:], stats=False)
    g1.close()
    rep["mode1"] = {"oracle_misclass_vs_truth": _misclass(m1, gt), "f16_misclass_vs_truth": _misclass(gm1, gt),
                    "f16_mask_agreement_with_oracle": float((gm1 == m1).mean())}
    # per-channel independent mixtures (COG_PERCHAN): oracle and FP16 GPU, reported
    o2 = oracle_run(params(W, H, K, flags=15 | 64))
    o2.train(frames[:NT])
    m2 = np.stack([o2.apply(frames[NT + t], want_stage=False, want_near=False)[0] for t in range(NF)])
    g2 = GpuRun(params(W, H, K, flags=15 | 64), "f16")
    g2.train(frames_d[:NT])
    gm2, _, _ = g2.apply(frames_d[NT:], stats=False)
    g2.close()
    rep["perchan"] = {"oracle_misclass_vs_truth": _misclass(m2, gt), "f16_misclass_vs_truth": _misclass(gm2, gt),
                      "f16_mask_agreement_with_oracle": float((gm2 == m2).mean())}
    rep["cog_f16_vs_plain_misclass_ratio"] = rep["f16"]["misclass_vs_truth"] / max(1e-12, rep["plain_gmm_f16_misclass_vs_truth"])
    REPORT[name] = rep
    if c["kind"] == "dynamic":
        assert rep["f16"]["misclass_vs_truth"] < rep["plain_gmm_f16_misclass_vs_truth"]
