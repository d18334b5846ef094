"""Test helper: one small run of every kernel family through the C ABI
(per-frame cascade with and without temporal sampling, the 4-bit prior,
the clip kernel, a batch of mixed streams, the plain mixture).  Run in a
process that loaded the COG_DEBUG library (COG_LIB_VARIANT=debug) it must
end with no failed bounds check; its masks must equal those of libcog.so.

    python tests/debug_build_workload.py OUT.npz
"""
from __future__ import annotations

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def run() -> dict:
    import torch

    from cogsynth import Scene
    from cogsynth.gpu import GpuScene
    from paper_1705_09339_gb300 import cog

    out = {}
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        st = s.cuda_stream

        def scene(w, h, seed, n):
            return GpuScene(Scene(w, h, seed, kind="dynamic", n_train=20, fg_frac=0.06, switch_at=8)).render(0, n)

        def ctx(w, h, k, dt, fr, **over):
            p = cog.cog_default_params(w, h, k, state_dtype=dt, **over)
            c = cog.cog_create(p, st)
            cog.cog_train_prior(c, fr[:20], 20)
            return c

        # per frame: a ragged size, K=5 FP16; temporal sampling; 4-bit prior
        for name, (w, h, k, dt, over) in {
                "frame": (333, 171, 5, "f16", {}),
                "sample": (256, 128, 3, "f32", {"flags": cog.COG_ALL | cog.COG_SAMPLE}),
                "prior4": (161, 97, 5, "bf16", {"kde_bits": 4})}.items():
            fr = scene(w, h, 3, 36)
            c = ctx(w, h, k, dt, fr, **over)
            m = torch.empty((16, h, w), dtype=torch.uint8, device="cuda")
            for t in range(16):
                cog.cog_apply(c, fr[20 + t], m[t])
            cog.cog_sync(c)
            out[name] = m.cpu().numpy()
            cog.cog_destroy(c)
        # clip of 16 frames
        w, h = 200, 120
        fr = scene(w, h, 5, 36)
        c = ctx(w, h, 5, "f16", fr)
        m = torch.empty((16, h, w), dtype=torch.uint8, device="cuda")
        cog.cog_apply_clip(c, fr[20:36], 16, m)
        cog.cog_sync(c)
        out["clip"] = m.cpu().numpy()
        # plain mixture
        m = torch.empty((4, h, w), dtype=torch.uint8, device="cuda")
        for t in range(4):
            cog.cog_apply_plain_gmm(c, fr[20 + t], m[t])
        cog.cog_sync(c)
        out["plain"] = m.cpu().numpy()
        cog.cog_destroy(c)
        # a batch of mixed streams: K 3/5, FP32/FP16, per-channel mixtures
        specs = [(160, 120, 3, "f32", {}), (97, 61, 5, "f16", {}),
                 (64, 48, 5, "f16", {"flags": cog.COG_ALL | cog.COG_PERCHAN})]
        frs = [scene(w_, h_, 10 + i, 26) for i, (w_, h_, _, _, _) in enumerate(specs)]
        cs = [ctx(w_, h_, k_, dt_, frs[i], **o_) for i, (w_, h_, k_, dt_, o_) in enumerate(specs)]
        b = cog.cog_batch_create(cs, st)
        ms = [torch.empty((6, h_, w_), dtype=torch.uint8, device="cuda") for (w_, h_, _, _, _) in specs]
        for t in range(6):
            cog.cog_batch_apply(b, [frs[i][20 + t] for i in range(len(specs))], [ms[i][t] for i in range(len(specs))])
        cog.cog_batch_sync(b)
        for i, c in enumerate(cs):
            cog.cog_sync(c)
            out[f"batch{i}"] = ms[i].cpu().numpy()
        cog.cog_batch_destroy(b)
        for c in cs:
            cog.cog_destroy(c)
    out["debug_build"] = np.array([cog.lib.cog_debug_build()])
    return out


if __name__ == "__main__":
    np.savez(sys.argv[1], **run())
