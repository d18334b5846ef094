"""Continuous-batching frame server: many cameras, one GPU.

Every admitted camera keeps its whole model (state buffer) resident in HBM
and owns two device frame slots and a mask buffer.  Frames arrive in host
memory at any time (`submit`).  The server loop repeatedly takes, for every
camera that has a frame waiting and a free slot, the oldest frame; copies
those frames to their slots on a copy stream; runs one batched cascade step
over exactly those cameras (`cog_batch_apply_active`: one replay of one
captured CUDA graph); and copies their masks back.  Frames that arrive while
a step is on the GPU join the next step, whose copies overlap the running
step.  A completion thread stamps each frame's latency from arrival to its
mask being in host memory.

Admission is by free device memory: a camera is admitted only if its state,
slots and masks fit in the memory left above a reserve.
"""
from __future__ import annotations

import collections
import threading
import time

import numpy as np

from . import cog


class Camera:
    def __init__(self, cid: int, width: int, height: int, K: int, dtype: str):
        self.id, self.width, self.height, self.K, self.dtype = cid, width, height, K, dtype
        self.P = width * height
        self.params = cog.cog_default_params(width, height, K, state_dtype=dtype)
        self.ctx = None
        self.slots = []          # two device frame buffers
        self.mask_dev = None
        self.mask_host = []      # two pinned host mask buffers
        self.pending = collections.deque()   # (host frame, arrival time, sequence number)
        self.inflight = 0        # frames on the device (at most 2: the two slots)
        self.done = 0            # frames completed
        self.seq = 0             # frames submitted


class FrameServer:
    def __init__(self, device=None, reserve_bytes: int = 4 << 30, keep_masks: bool = False):
        import torch
        self.torch = torch
        self.dev = torch.device(device or "cuda")
        self.compute = torch.cuda.Stream(self.dev)
        self.copy = torch.cuda.Stream(self.dev)
        self.reserve = reserve_bytes
        self.cameras: list[Camera] = []
        self.refused: list[tuple] = []
        self.batch = None
        self.lock = threading.Lock()
        self.cv = threading.Condition(self.lock)
        self.latencies = []
        self.frames_done = 0
        self.pixels_done = 0
        self.steps = 0
        self.keep_masks = keep_masks
        self.results = collections.defaultdict(list)   # camera id -> masks (keep_masks)
        self._stop = False
        self._completions = collections.deque()
        self._comp_cv = threading.Condition()

    # ------------------------------------------------------------ admission
    def admit(self, width: int, height: int, K: int, dtype: str, train_frames) -> Camera | None:
        """Admits a camera if its resident model and buffers fit in free
        device memory above the reserve, and trains it on train_frames (a
        device uint8 tensor [N, H, W, 3]).  Returns None when refused."""
        torch = self.torch
        cam = Camera(len(self.cameras), width, height, K, dtype)
        need = cog.cog_state_bytes(cam.params) + 2 * cam.P * 3 + cam.P + (1 << 20)
        free, _ = torch.cuda.mem_get_info(self.dev)
        if free - need < self.reserve:
            self.refused.append((width, height, K, dtype, need))
            return None
        cam.ctx = cog.cog_create(cam.params, self.compute.cuda_stream)
        cam.slots = [torch.empty((height, width, 3), dtype=torch.uint8, device=self.dev) for _ in range(2)]
        cam.mask_dev = [torch.empty((height, width), dtype=torch.uint8, device=self.dev) for _ in range(2)]
        cam.mask_host = [torch.empty((height, width), dtype=torch.uint8).pin_memory() for _ in range(2)]
        with torch.cuda.stream(self.compute):
            cog.cog_train_prior(cam.ctx, train_frames, train_frames.shape[0])
        cog.cog_sync(cam.ctx)
        self.cameras.append(cam)
        return cam

    def start(self):
        """Builds the batch over the admitted cameras and starts the loop."""
        self.batch = cog.cog_batch_create([c.ctx for c in self.cameras], self.compute.cuda_stream)
        self._loop_t = threading.Thread(target=self._loop, daemon=True)
        self._done_t = threading.Thread(target=self._completer, daemon=True)
        self._t0 = time.perf_counter()
        self._loop_t.start()
        self._done_t.start()

    def submit(self, cam: Camera, frame_host, t_arrival: float | None = None):
        """Queues a host frame (pinned uint8 tensor [H, W, 3]) for cam."""
        with self.cv:
            cam.pending.append((frame_host, time.perf_counter() if t_arrival is None else t_arrival, cam.seq))
            cam.seq += 1
            self.cv.notify()

    # ------------------------------------------------------------ the loop
    def _loop(self):
        torch = self.torch
        n = len(self.cameras)
        while True:
            with self.cv:
                while not self._stop and not any(c.pending and c.inflight < 2 for c in self.cameras):
                    self.cv.wait(timeout=0.05)
                if self._stop and not any(c.pending for c in self.cameras):
                    break
                picks = []
                for c in self.cameras:
                    if c.pending and c.inflight < 2:
                        picks.append((c, c.pending.popleft()))
                        c.inflight += 1
            if not picks:
                continue
            active = np.zeros(n, np.uint8)
            frames = [None] * n
            masks = [None] * n
            tick = []
            with torch.cuda.stream(self.copy):
                for c, (fh, ta, sq) in picks:
                    s = sq % 2
                    c.slots[s].copy_(fh, non_blocking=True)
                    active[c.id] = 1
                    frames[c.id] = c.slots[s]
                    masks[c.id] = c.mask_dev[s]
                    tick.append((c, ta, sq, s))
                copied = torch.cuda.Event()
                copied.record(self.copy)
            self.compute.wait_event(copied)
            cog.cog_batch_apply_active(self.batch, frames, masks, active)
            applied = torch.cuda.Event()
            applied.record(self.compute)
            self.copy.wait_event(applied)
            with torch.cuda.stream(self.copy):
                for c, ta, sq, s in tick:
                    c.mask_host[s].copy_(c.mask_dev[s], non_blocking=True)
                ready = torch.cuda.Event()
                ready.record(self.copy)
            self.steps += 1
            with self._comp_cv:
                self._completions.append((ready, tick))
                self._comp_cv.notify()
        with self._comp_cv:
            self._completions.append(None)
            self._comp_cv.notify()

    def _completer(self):
        while True:
            with self._comp_cv:
                while not self._completions:
                    self._comp_cv.wait()
                item = self._completions.popleft()
            if item is None:
                return
            ready, tick = item
            ready.synchronize()
            t = time.perf_counter()
            with self.cv:
                for c, ta, sq, s in tick:
                    self.latencies.append(t - ta)
                    self.frames_done += 1
                    self.pixels_done += c.P
                    c.inflight -= 1
                    c.done += 1
                    if self.keep_masks:
                        self.results[c.id].append((sq, c.mask_host[s].numpy().copy()))
                self.cv.notify()

    def stop(self):
        """Drains every queued frame, stops the threads and returns the
        serving statistics."""
        with self.cv:
            self._stop = True
            self.cv.notify()
        self._loop_t.join()
        self._done_t.join()
        wall = time.perf_counter() - self._t0
        lat = np.array(self.latencies) * 1e3
        cog.cog_batch_sync(self.batch)
        return {"frames": self.frames_done, "steps": self.steps, "wall_s": round(wall, 3),
                "mpixel_per_s": round(self.pixels_done / wall / 1e6, 1),
                "latency_ms": {"p50": round(float(np.percentile(lat, 50)), 3) if lat.size else None,
                               "p99": round(float(np.percentile(lat, 99)), 3) if lat.size else None,
                               "max": round(float(lat.max()), 3) if lat.size else None},
                "cameras": len(self.cameras), "refused": len(self.refused)}

    def close(self):
        if self.batch is not None:
            cog.cog_batch_destroy(self.batch)
            self.batch = None
        for c in self.cameras:
            cog.cog_destroy(c.ctx)
        self.cameras = []
