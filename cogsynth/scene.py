"""Synthetic scenes shaped like the paper's surveillance workloads.

The paper evaluates on the Wallflower videos and CDW-2014, neither of which
is available; these scenes stand in for them.  Everything is integer and
counter-based: the value of channel c of pixel p in frame t depends only on
(seed, stream, t, p, c), so any subset of pixels or frames can be rendered
independently and the CUDA twin reproduces it bit for bit.

Scene kinds
-----------
``rects``   static smooth texture + per-pixel camera noise; in test frames
            three constant-colour rectangles (10-30 px) moving at 1-3 px per
            frame with bouncing, and a linear brightness ramp of +20 levels
            over 300 frames.
``dynamic`` the same texture and noise, plus dynamic background: discs
            covering about 10 % of the pixels that flip to a second colour
            mode with probability 0.3 per frame, a region whose level sways
            by 8 sin(2 pi t / 20); in test frames eight random-walk ellipses
            covering a chosen foreground fraction, and a sudden +60 light
            switch at a chosen test frame.

Noise: sigma_p ~ U(2, 6) fixed per pixel; per frame an Irwin-Hall sum of
four 16-bit uniforms (one splitmix64 draw) scaled to sigma_p, rounded with
integer division, and the value clipped to [0, 255].
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1
GOLD = 0x9E3779B97F4A7C15

# hash tags
TAG_BG, TAG_SIG, TAG_NOISE, TAG_BLOB, TAG_BMODE = 1, 2, 3, 4, 5
TAG_SWAY, TAG_ELL, TAG_WALK, TAG_RECT = 6, 7, 8, 9

NOISE_DEN = 605395          # 16 * sigma of a sum of four 16-bit uniforms
NOISE_MEAN = 131070         # mean of that sum
NOISE_BIAS = 64             # keeps the rounded division's numerator positive
GRID = 16                   # texture cell size in pixels
MAX_OBJ = 16
MAX_BLOBS = 256

_U64 = np.uint64


def sm64(x):
    """splitmix64 finaliser (Steele, Lea, Flood 2014) on python ints or
    numpy uint64 arrays."""
    if isinstance(x, np.ndarray):
        z = x + _U64(GOLD)
        z = (z ^ (z >> _U64(30))) * _U64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> _U64(27))) * _U64(0x94D049BB133111EB)
        return z ^ (z >> _U64(31))
    z = (x + GOLD) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def _key(seed: int, stream: int, tag: int, a: int = 0) -> int:
    k = sm64(seed & MASK64)
    k = sm64(k ^ (((stream + 1) * GOLD) & MASK64))
    return sm64(k ^ ((tag << 48) | (a & ((1 << 48) - 1))))


def _h(base: int, i: int) -> int:
    return sm64(base ^ (i & MASK64))


@dataclass
class Scene:
    width: int
    height: int
    seed: int
    stream: int = 0
    kind: str = "rects"          # "rects" | "dynamic"
    n_train: int = 200
    fg_frac: float = 0.02        # dynamic: ellipse foreground fraction
    switch_at: int = 600         # dynamic: test frame of the +60 light switch
    switch_amp: int = 60
    ramp_amp: int = 20           # rects: brightness ramp over ramp_len frames
    ramp_len: int = 300
    n_ellipses: int = 8
    _walk: list = field(default_factory=list, repr=False)

    def __post_init__(self):
        W, H = self.width, self.height
        self.P = W * H
        s, st = self.seed, self.stream
        # smooth texture: bilinear value noise on a 16-px grid, levels 40..215
        gw, gh = W // GRID + 2, H // GRID + 2
        gy, gx, c = np.meshgrid(np.arange(gh, dtype=np.uint64), np.arange(gw, dtype=np.uint64),
                                np.arange(3, dtype=np.uint64), indexing="ij")
        idx = (((gy << _U64(20)) | gx) << _U64(2)) | c
        grid = (40 + (sm64(idx ^ _U64(_key(s, st, TAG_BG))) % _U64(176))).astype(np.int64)
        y = np.arange(H, dtype=np.int64)[:, None]
        x = np.arange(W, dtype=np.int64)[None, :]
        cy, fy = y // GRID, y % GRID
        cx, fx = x // GRID, x % GRID
        g00 = grid[cy, cx]
        g10 = grid[cy, cx + 1]
        g01 = grid[cy + 1, cx]
        g11 = grid[cy + 1, cx + 1]
        w00 = ((GRID - fx) * (GRID - fy))[..., None]
        w10 = (fx * (GRID - fy))[..., None]
        w01 = ((GRID - fx) * fy)[..., None]
        w11 = (fx * fy)[..., None]
        bg = (g00 * w00 + g10 * w10 + g01 * w01 + g11 * w11 + GRID * GRID // 2) // (GRID * GRID)
        self.bg = bg.reshape(self.P, 3).astype(np.int16)
        # per-pixel noise level sigma_p = sig16 / 16 in [2, 6]
        p = np.arange(self.P, dtype=np.uint64)
        self.sig16 = (32 + sm64(p ^ _U64(_key(s, st, TAG_SIG))) % _U64(65)).astype(np.int32)
        self.blob_id = np.full(self.P, -1, np.int32)
        self.blob_delta = np.zeros((0, 3), np.int16)
        self.sway_rect = (0, 0, 0, 0)
        if self.kind == "dynamic":
            self._init_dynamic()
        elif self.kind != "rects":
            raise ValueError(f"unknown scene kind {self.kind}")
        self._init_objects()

    # ---------------------------------------------------------------- static
    def _init_dynamic(self):
        W, H = self.width, self.height
        kb = _key(self.seed, self.stream, TAG_BLOB)
        r = max(4, W // 40)
        nb = min(MAX_BLOBS, max(1, int(round(0.10 * self.P / (math.pi * r * r)))))
        delta = np.zeros((nb, 3), np.int16)
        bid = np.full((H, W), -1, np.int32)
        for b in reversed(range(nb)):           # lower index wins on overlap
            cx = _h(kb, b * 8 + 0) % W
            cy = _h(kb, b * 8 + 1) % H
            for c in range(3):
                hv = _h(kb, b * 8 + 2 + c)
                mag = 40 + (hv >> 8) % 41
                delta[b, c] = mag if (hv & 1) else -mag
            x0, x1 = max(0, cx - r), min(W, cx + r + 1)
            y0, y1 = max(0, cy - r), min(H, cy + r + 1)
            yy, xx = np.mgrid[y0:y1, x0:x1]
            inside = (xx - cx) ** 2 + (yy - cy) ** 2 <= r * r
            sub = bid[y0:y1, x0:x1]
            sub[inside] = b
        self.blob_id = bid.reshape(-1)
        self.blob_delta = delta
        ks = _key(self.seed, self.stream, TAG_SWAY)
        sw, sh = max(1, W // 4), max(1, H // 4)
        x0 = _h(ks, 0) % (W - sw + 1)
        y0 = _h(ks, 1) % (H - sh + 1)
        self.sway_rect = (x0, y0, x0 + sw, y0 + sh)

    def _init_objects(self):
        W, H = self.width, self.height
        if self.kind == "rects":
            kr = _key(self.seed, self.stream, TAG_RECT)
            self.rects = []
            for i in range(3):
                f = lambda j: _h(kr, i * 16 + j)  # noqa: E731
                w, h = 10 + f(0) % 21, 10 + f(1) % 21
                w, h = min(w, W), min(h, H)
                col = (f(2) % 256, f(3) % 256, f(4) % 256)
                vx = (1 + f(5) % 3) * (1 if f(6) & 1 else -1)
                vy = (1 + f(7) % 3) * (1 if f(8) & 1 else -1)
                x0, y0 = f(9) % (W - w + 1), f(10) % (H - h + 1)
                self.rects.append((w, h, col, vx, vy, x0, y0))
        else:
            ke = _key(self.seed, self.stream, TAG_ELL)
            area = self.fg_frac * self.P / self.n_ellipses
            self.ells = []
            for e in range(self.n_ellipses):
                f = lambda j: _h(ke, e * 16 + j)  # noqa: E731
                rho = 0.5 + (f(0) % 1501) / 1000.0
                a = max(2, int(round(math.sqrt(area * rho / math.pi))))
                b = max(2, int(round(area / (math.pi * a))))
                col = (f(1) % 256, f(2) % 256, f(3) % 256)
                self.ells.append([a, b, col, f(4) % W, f(5) % H])
            self._walk = [[(e[3], e[4]) for e in self.ells]]

    # ------------------------------------------------------------- per frame
    def _ellipse_pos(self, n: int):
        kw = _key(self.seed, self.stream, TAG_WALK)
        W, H = self.width, self.height
        while len(self._walk) <= n:
            m = len(self._walk) - 1
            cur = []
            for e, (x, y) in enumerate(self._walk[-1]):
                hv = _h(kw, m * 64 + e)
                x += int(hv % 7) - 3
                y += int((hv >> 8) % 7) - 3
                if x < 0:
                    x = -x
                if x > W - 1:
                    x = 2 * (W - 1) - x
                if y < 0:
                    y = -y
                if y > H - 1:
                    y = 2 * (H - 1) - y
                cur.append((x, y))
            self._walk.append(cur)
        return self._walk[n]

    def frame_desc(self, t: int) -> dict:
        """Per-frame scene parameters for global frame index t (training
        frames are t < n_train)."""
        n = t - self.n_train
        objs = []
        offset = sway = 0
        modes = np.zeros(len(self.blob_delta), bool)
        if self.kind == "rects":
            if n >= 0:
                nn = min(n, self.ramp_len - 1)
                offset = (self.ramp_amp * nn + (self.ramp_len - 1) // 2) // (self.ramp_len - 1)
                for (w, h, col, vx, vy, x0, y0) in self.rects:
                    x = _bounce(x0 + vx * n, self.width - w)
                    y = _bounce(y0 + vy * n, self.height - h)
                    objs.append((0, x, y, x + w, y + h) + col)
        else:
            kb = _key(self.seed, self.stream, TAG_BMODE, t)
            modes = np.array([_h(kb, b) % 1000 < 300 for b in range(len(self.blob_delta))], bool)
            sway = int(math.floor(8.0 * math.sin(2.0 * math.pi * t / 20.0) + 0.5))
            if n >= 0:
                if n >= self.switch_at:
                    offset = self.switch_amp
                for (a, b, col, _, _), (x, y) in zip(self.ells, self._ellipse_pos(n)):
                    objs.append((1, x, y, a, b) + col)
        return dict(noise_base=_key(self.seed, self.stream, TAG_NOISE, t), offset=offset,
                    sway=sway, modes=modes, objects=objs[:MAX_OBJ])

    def render(self, t: int, pix: np.ndarray | None = None):
        """Render global frame t.  Returns (values[n, 3] uint8, gt[n] uint8)
        for the pixel indices ``pix`` (all pixels when None)."""
        d = self.frame_desc(t)
        if pix is None:
            pix = np.arange(self.P, dtype=np.int64)
        pix = np.asarray(pix, dtype=np.int64)
        x = pix % self.width
        y = pix // self.width
        base = self.bg[pix].astype(np.int64)
        if len(self.blob_delta):
            bid = self.blob_id[pix]
            on = bid >= 0
            on[on] = d["modes"][bid[on]]
            base[on] += self.blob_delta[bid[on]]
            x0, y0, x1, y1 = self.sway_rect
            inr = (x >= x0) & (x < x1) & (y >= y0) & (y < y1)
            base[inr] += d["sway"]
        gt = np.zeros(len(pix), bool)
        for (kind, a0, b0, a1, b1, r, g, b) in d["objects"]:
            if kind == 0:
                ins = (x >= a0) & (x < a1) & (y >= b0) & (y < b1)
            else:
                dx, dy = x - a0, y - b0
                ins = (dx * b1) ** 2 + (dy * a1) ** 2 <= (a1 * b1) ** 2
            base[ins] = (r, g, b)
            gt |= ins
        base += d["offset"]
        idx = (pix.astype(np.uint64)[:, None] << _U64(2)) | np.arange(3, dtype=np.uint64)[None, :]
        u = sm64(idx ^ _U64(d["noise_base"]))
        m16 = _U64(0xFFFF)
        s = ((u & m16) + ((u >> _U64(16)) & m16) + ((u >> _U64(32)) & m16) + (u >> _U64(48)))
        z = s.astype(np.int64) - NOISE_MEAN
        noise = (z * self.sig16[pix].astype(np.int64)[:, None] + NOISE_DEN // 2
                 + NOISE_BIAS * NOISE_DEN) // NOISE_DEN - NOISE_BIAS
        v = np.clip(base + noise, 0, 255).astype(np.uint8)
        return v, (gt * 255).astype(np.uint8)

    def frames(self, t0: int, n: int, pix: np.ndarray | None = None):
        """Frames t0..t0+n-1 as [n, npix, 3] uint8 plus ground truth [n, npix]."""
        vs, gs = zip(*(self.render(t, pix) for t in range(t0, t0 + n)))
        return np.stack(vs), np.stack(gs)


def _bounce(u: int, L: int) -> int:
    if L <= 0:
        return 0
    u %= 2 * L
    return u if u <= L else 2 * L - u


# --------------------------------------------------------------------------
# Named workloads (sizes, lengths and scene kinds of the five benchmark
# configurations; the first three are single streams).
# --------------------------------------------------------------------------
def workload(name: str, fg_frac: float = 0.02, seed: int | None = None) -> dict:
    """Scene, model size and run length of a named workload."""
    if name == "qvga_rects":        # 160x120, K=3, FP32 state
        sc = Scene(160, 120, 1 if seed is None else seed, kind="rects", n_train=200)
        return dict(scene=sc, K=3, n_train=200, n_test=300, dtype="f32")
    if name == "vga_dynamic":       # 640x480, K=5
        sc = Scene(640, 480, 2 if seed is None else seed, kind="dynamic", n_train=500,
                   fg_frac=fg_frac, switch_at=600)
        return dict(scene=sc, K=5, n_train=500, n_test=1000, dtype="f32")
    if name == "hd_dynamic":        # 1920x1080, K=5, FP16 state
        sc = Scene(1920, 1080, 3 if seed is None else seed, kind="dynamic", n_train=500,
                   fg_frac=fg_frac, switch_at=600)
        return dict(scene=sc, K=5, n_train=500, n_test=2000, dtype="f16")
    raise KeyError(name)
