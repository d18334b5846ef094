"""Launch-shape autotuner for the two cascade kernels.

The shape of a cascade launch -- threads per stage-0/1 CTA, threads per
mixture-stage CTA, mixture-stage CTAs per SM -- changes speed but not
results.  The best shape depends on the frame size, K, the storage type and
how many pixels survive to the mixture stage.  The tuner measures every
candidate on a scratch context trained on the caller's frames, over the
caller's own test frames, with CUDA events and an L2 flush between frames,
and caches the winner per (GPU, frame size, K, storage type).
"""
from __future__ import annotations

import json
import os
import threading

from . import cog

CANDIDATES = [(k1, k2, ps) for k1 in (64, 128, 256) for k2 in (64, 128) for ps in (0, 4, 8)]
DEFAULT = (128, 64, 0)
_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tune_cache.json")
_lock = threading.Lock()


def _key(p: cog.cog_params, device_name: str) -> str:
    dt = {cog.COG_F32: "f32", cog.COG_F16: "f16", cog.COG_BF16: "bf16"}[p.state_dtype]
    return f"{device_name}|{p.width}x{p.height}|K{p.K}|{dt}|flags{p.flags}"


def load_cache(path: str = _CACHE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def cached(p: cog.cog_params, path: str = _CACHE):
    import torch
    return load_cache(path).get(_key(p, torch.cuda.get_device_name()))


def tune(p: cog.cog_params, train, test, n_frames: int = 12, warmup: int = 3, path: str | None = _CACHE,
         candidates=CANDIDATES) -> dict:
    """Times each candidate shape on a scratch context.

    train: device uint8 tensor [N, H, W, 3] of training frames; test: device
    tensor [M, H, W, 3] with M >= warmup + n_frames.  Returns
    {"best": (k1, k2, per_sm), "us": {shape: mean step microseconds}} and
    stores the best shape in the cache at `path` (None: no cache)."""
    import torch
    assert test.shape[0] >= warmup + n_frames
    stream = torch.cuda.current_stream()
    ctx = cog.cog_create(p, stream.cuda_stream)
    try:
        cog.cog_train_prior(ctx, train, train.shape[0])
        mask = torch.empty(test.shape[1:3], dtype=torch.uint8, device=test.device)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=test.device)
        res = {}
        for cand in candidates:
            cog.cog_set_launch(ctx, *cand)
            for i in range(warmup):
                cog.cog_apply(ctx, test[i], mask)
            ev = []
            for i in range(n_frames):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                cog.cog_apply(ctx, test[warmup + i], mask)
                b.record(stream)
                ev.append((a, b))
            torch.cuda.synchronize()
            res[cand] = 1e3 * sum(a.elapsed_time(b) for a, b in ev) / n_frames
    finally:
        cog.cog_destroy(ctx)
    best = min(res, key=res.get)
    out = {"best": best, "us": {f"{k[0]}/{k[1]}/{k[2]}": round(v, 2) for k, v in res.items()}}
    if path:
        with _lock:
            c = load_cache(path)
            c[_key(p, torch.cuda.get_device_name())] = {"shape": list(best), "us": out["us"]}
            tmp = path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(c, f, indent=1)
            os.replace(tmp, path)
    return out


def apply_best(ctx, p: cog.cog_params, path: str = _CACHE) -> tuple:
    """Sets the cached best shape on ctx (the default shape when none is
    cached) and returns it."""
    e = cached(p, path)
    shape = tuple(e["shape"]) if e else DEFAULT
    cog.cog_set_launch(ctx, *shape)
    return shape
