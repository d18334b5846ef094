"""Test harness: runs the CUDA path (through the C ABI) and the FP64 oracle
on the same seeded inputs and compares them.  Test code only."""
from __future__ import annotations

import numpy as np

# parameter values shared by both sides, rounded to what the FP32 library
# actually receives so the two compute with identical constants
BASE = dict(alpha=0.01, lambda_=2.5, T_bg=0.7, w_init=0.05, var_init=225.0, var_min=4.0,
            var_max=900.0, tau_fd=8.0, eta=0.125, c_halt=0.9, w_illum=0.75, q_null=13, kde_bw=4,
            r1=10, r2=30, illum_permille=700, flags=15, c_skip=0.95, skip_period=4, kde_bits=8)
FLOATS = ("alpha", "lambda_", "T_bg", "w_init", "var_init", "var_min", "var_max", "tau_fd", "eta",
          "c_halt", "w_illum", "c_skip")


def params(W, H, K, **over):
    d = dict(BASE, width=W, height=H, K=K)
    d.update(over)
    for k in FLOATS:
        d[k] = float(np.float32(d[k]))
    return d


def to_cog(d, dtype="f32"):
    from paper_1705_09339_gb300 import cog
    p = cog.cog_default_params(d["width"], d["height"], d["K"], state_dtype=dtype)
    for k, v in d.items():
        if k in ("width", "height", "K"):
            continue
        setattr(p, "eta_conf" if k == "eta" else k, v)
    return p


class GpuRun:
    """One CUDA-path context over a stream of frames."""

    def __init__(self, d, dtype="f32", device="cuda"):
        import torch
        from paper_1705_09339_gb300 import cog
        self.torch, self.cog = torch, cog
        self.d, self.dtype = d, dtype
        self.W, self.H = d["width"], d["height"]
        self.P = self.W * self.H
        self.dev = torch.device(device)
        self.p = to_cog(d, dtype)
        self.ctx = cog.cog_create(self.p, torch.cuda.current_stream().cuda_stream)

    def train(self, frames):
        t = self._dev_frames(frames)
        self.cog.cog_train_prior(self.ctx, t, t.shape[0])

    def _dev_frames(self, frames):
        torch = self.torch
        if isinstance(frames, np.ndarray):
            return torch.from_numpy(np.ascontiguousarray(frames).reshape(-1, self.H, self.W, 3)).to(self.dev)
        return frames

    def apply(self, frames, stats=True, plain=False):
        """Applies frames [n, P, 3] (numpy or device tensor); returns masks,
        stage maps [n, P] and per-frame stats."""
        torch = self.torch
        fr = self._dev_frames(frames)
        n = fr.shape[0]
        masks = torch.empty((n, self.P), dtype=torch.uint8, device=self.dev)
        stages = torch.empty((n, self.P), dtype=torch.uint8, device=self.dev)
        st = []
        for i in range(n):
            if plain:
                self.cog.cog_apply_plain_gmm(self.ctx, fr[i], masks[i])
            else:
                st.append(self.cog.cog_apply(self.ctx, fr[i], masks[i], stages[i], want_stats=stats))
        self.cog.cog_sync(self.ctx)
        return masks.cpu().numpy(), stages.cpu().numpy(), st

    def state(self):
        raw = self.cog.cog_export_state(self.ctx, self.p)
        return self.cog.decode_state(raw, self.p)

    def set_state(self, st):
        raw = self.cog.cog_export_state(self.ctx, self.p)
        self.cog.cog_import_state(self.ctx, self.cog.encode_state(raw, self.p, st))

    def close(self):
        self.cog.cog_destroy(self.ctx)


def oracle_run(d):
    import oracle
    return oracle.Oracle(d)


def rel_err(a, b):
    return np.abs(a - b) / np.maximum(np.abs(b), 1.0)


def compare_stream(gm, gs, om, os_, near):
    """Masks and stage maps [n, P] of both sides plus the oracle's near
    record; returns (agreement, unexplained mismatches, ever_near)."""
    ever = np.zeros(gm.shape[1], bool)
    unexplained = 0
    for t in range(gm.shape[0]):
        ever |= near[t] != 0
        bad = (gm[t] != om[t]) | (gs[t] != os_[t])
        unexplained += int((bad & ~ever).sum())
    agree = float((gm == om).mean())
    return agree, unexplained, ever


def state_errors(g, o, mask):
    """Largest relative error of each model field over the pixels in mask."""
    out = {}
    for k in ("w", "mu", "var", "rga_m", "rga_v", "conf", "wc"):
        if k not in g:
            continue
        a, b = g[k][mask], o[k][mask]
        out[k] = float(rel_err(a, b).max()) if a.size else 0.0
    for k in ("label", "prev", "qa", "qb"):
        out[k] = int((g[k][mask] != o[k][mask]).sum())
    return out


def oracle_state(o):
    s = o.state
    return dict(w=s.w, mu=s.mu, var=s.var, rga_m=s.rga_m, rga_v=s.rga_v, conf=s.conf, label=s.label,
                prev=s.prev, kde=s.kde, qa=s.qa, qb=s.qb, top=s.top, wc=s.wc)


def random_state(rng, P, K, dtype="f32", fg_frac=0.2, mode1=False, perchan=False, kde_bits=8, kde_const=None):
    """A seeded model state with the value ranges the method produces,
    rounded to the storage type so both sides start from the same values."""
    q = {"f32": np.float32, "f16": np.float16, "bf16": None}[dtype]

    def r(x):
        x = np.asarray(x, np.float64)
        if dtype == "bf16":
            f = x.astype(np.float32).view(np.uint32)
            f = ((f + 0x7FFF + ((f >> 16) & 1)) >> 16) << 16
            return f.astype(np.uint32).view(np.float32).astype(np.float64)
        return x.astype(q).astype(np.float64)

    w = rng.gamma(0.7, size=(P, K))
    w[rng.random((P, K)) < 0.25] = 0.0
    w[:, 0] += 1e-3
    w = w / w.sum(axis=1, keepdims=True)
    mu = rng.uniform(0, 255, (P, K, 3))
    var = np.exp(rng.uniform(np.log(4.0), np.log(900.0), (P, K, 3)))
    rga_m = rng.uniform(0, 255, (P, 3))
    rga_v = np.exp(rng.uniform(np.log(4.0), np.log(900.0), (P, 3)))
    conf = rng.uniform(0, 1, P)
    qa = rng.integers(0, 256, P)
    qb = np.minimum(rng.integers(0, 256, P), 255 - qa)
    if kde_const is not None:
        # one level everywhere (large frames: no random table of P x 768)
        kde = np.full((P, 3, 256), kde_const, np.uint8)
    elif kde_bits == 4:
        # levels of 15; level 0 (17 * 0 < q_null = 13) is the nullified one
        kde = rng.integers(0, 16, (P, 3, 256)).astype(np.uint8)
        kde[rng.random((P, 3, 256)) < 0.3] = 0
    else:
        kde = rng.integers(0, 256, (P, 3, 256)).astype(np.uint8)
        kde[rng.random((P, 3, 256)) < 0.3] = rng.integers(0, 13)
    prev = rng.integers(0, 256, (P, 3)).astype(np.uint8)
    label = (rng.random(P) < fg_frac).astype(np.uint8)
    # COG_MODE1 keeps the stage-1 record equal to the rank-1 mode it mirrors
    key = w ** 2 / var.mean(axis=2)
    top = np.argmax(key, axis=1).astype(np.uint8)
    st = dict(w=r(w), mu=r(mu), var=r(var), rga_m=r(rga_m), rga_v=r(rga_v), conf=r(conf),
              label=label, prev=prev, kde=kde, qa=qa.astype(np.uint8), qb=qb.astype(np.uint8), top=top)
    if mode1:
        st["rga_m"] = st["mu"][np.arange(P), top].copy()
        st["rga_v"] = st["var"][np.arange(P), top].copy()
    if perchan:
        wc = rng.gamma(0.7, size=(P, 3, K))
        wc[rng.random((P, 3, K)) < 0.25] = 0.0
        wc[:, :, 0] += 1e-3
        st["wc"] = r(wc / wc.sum(axis=2, keepdims=True))
    return st


def random_frame(rng, st, mix=(0.4, 0.3, 0.3)):
    """A frame whose pixels repeat the previous value (stage 0 material),
    sit near a random model mode (stages 1/2), or are arbitrary."""
    P = st["prev"].shape[0]
    u = rng.random(P)
    f = rng.integers(0, 256, (P, 3))
    rep = u < mix[0]
    f[rep] = np.clip(st["prev"][rep].astype(int) + rng.integers(-6, 7, (int(rep.sum()), 3)), 0, 255)
    near = (u >= mix[0]) & (u < mix[0] + mix[1])
    k = rng.integers(0, st["mu"].shape[1], P)
    m = st["mu"][np.arange(P), k]
    sd = np.sqrt(st["var"][np.arange(P), k])
    g = np.clip(np.rint(m + rng.normal(0, 1, (P, 3)) * sd * 1.5), 0, 255).astype(int)
    f[near] = g[near]
    return f.astype(np.uint8)


def set_oracle_state(o, st):
    s = o.state
    for k in ("w", "mu", "var", "rga_m", "rga_v", "conf", "label", "prev", "kde", "qa", "qb", "top", "wc"):
        if k in st:
            getattr(s, k)[...] = st[k]
    s.illum[:] = 0
