"""Continuous-batching frame server: many cameras, one GPU.

Every admitted camera keeps its whole model (state buffer) resident in HBM.
Admission is by free device memory: a camera is admitted only if its state,
its two device frame slots and two mask slots fit in the memory left above
a reserve.  `start` hands the admitted cameras to the native server
(cog_server_*): a C++ worker thread repeatedly takes, for every camera that
has a frame waiting and a free slot, the oldest frame; uploads those frames
on a copy stream; runs one batched cascade step over exactly those cameras
(one replay of one captured CUDA graph); and downloads their masks.  Frames
that arrive while a step is on the GPU join the next step, whose uploads
overlap the running step.  A C++ completion thread stamps each frame's
latency from submission to its mask being in host memory.  Cameras join and
leave a running server between steps; a camera that leaves frees its HBM for
the next admission, which takes its index.  Python only admits cameras,
retires them and submits frames.
"""
from __future__ import annotations

import collections

import numpy as np

from . import cog


class PinnedArena:
    """Page-locked host memory handed out from a few large blocks, either of
    cog_host_alloc (kind "registered": huge-page memory locked with
    cudaHostRegister) or of cudaHostAlloc (kind "hostalloc", through torch).
    On the GB300's Grace host, host-to-device copies out of registered
    huge-page memory keep 160-180 GB/s from the first use, where
    cudaHostAlloc memory ran at 4-90 GB/s from box to box and stalled single
    uploads for tens of milliseconds."""

    def __init__(self, chunk_bytes: int = 1 << 30, kind: str = "registered"):
        import ctypes
        import torch
        assert kind in ("registered", "hostalloc")
        self.torch, self.ctypes = torch, ctypes
        self.chunk = chunk_bytes
        self.kind = kind
        self.blocks = []         # (address or None, tensor over the block)
        self.off = 0

    def _grow(self, n):
        torch, ctypes = self.torch, self.ctypes
        if self.kind == "registered":
            addr = cog.cog_host_alloc(n)
            arr = np.ctypeslib.as_array(ctypes.cast(addr, ctypes.POINTER(ctypes.c_uint8)), shape=(n,))
            self.blocks.append((addr, torch.from_numpy(arr)))
        else:
            self.blocks.append((None, torch.empty(n, dtype=torch.uint8, pin_memory=True)))
        self.off = 0

    def reserve(self, nbytes: int):
        """Allocates now one block that holds nbytes more, so that buffers
        taken next come from one large block.  Take it after the process's
        large device allocations: blocks locked before them copied at a few
        GB/s in some processes, blocks locked after them at 150-180 GB/s."""
        if not self.blocks or self.off + nbytes > self.blocks[-1][1].numel():
            self._grow(max(self.chunk, nbytes))

    def take(self, shape, dtype=None):
        """A page-locked tensor of `shape` (uint8 unless given), 256-byte
        aligned, valid until release()."""
        torch = self.torch
        dtype = dtype or torch.uint8
        nbytes = int(np.prod(shape)) * torch.empty((), dtype=dtype).element_size()
        span = (nbytes + 255) // 256 * 256
        if not self.blocks or self.off + span > self.blocks[-1][1].numel():
            self._grow(max(self.chunk, span))
        t = self.blocks[-1][1][self.off:self.off + nbytes]
        self.off += span
        return t.view(dtype).view(shape)

    def release(self):
        """Frees every block; no tensor from take() may be used afterwards."""
        for addr, _ in self.blocks:
            if addr is not None:
                cog.cog_host_free(addr)
        self.blocks = []
        self.off = 0


class Camera:
    def __init__(self, cid: int, width: int, height: int, K: int, dtype: str):
        self.id, self.width, self.height, self.K, self.dtype = cid, width, height, K, dtype
        self.P = width * height
        self.params = cog.cog_default_params(width, height, K, state_dtype=dtype)
        self.ctx = None
        self.seq = 0             # frames submitted
        self.mask_ring = []      # pinned host masks reused when results are not kept
        self.masks = []          # (seq, host mask) of every frame, when results are kept


class FrameServer:
    RING = 4                     # host mask buffers per camera when results are not kept
    # with keep_masks, results[camera index] lists (seq, mask) of the camera
    # now at that index (a camera that left keeps its own in Camera.masks)

    def __init__(self, device=None, reserve_bytes: int = 4 << 30, keep_masks: bool = False,
                 frame_memory: str = "registered", mask_memory: str = "hostalloc"):
        import torch
        self.torch = torch
        self.dev = torch.device(device or "cuda")
        self.reserve = reserve_bytes
        self.cameras: list[Camera | None] = []   # by stream index; None: the camera left
        self.refused: list[tuple] = []
        self.keep_masks = keep_masks
        # callers take their frame buffers from `arena`; the mask rings come
        # from `mask_arena`
        self.arena = PinnedArena(kind=frame_memory)
        self.mask_arena = PinnedArena(kind=mask_memory)
        self.results = collections.defaultdict(list)   # camera id -> (seq, mask) when keep_masks
        self._keep = []          # host buffers referenced by queued frames
        self.srv = None

    # ------------------------------------------------------------ admission
    def admit(self, width: int, height: int, K: int, dtype: str, train_frames) -> Camera | None:
        """Admits a camera if its resident model and buffers fit in free
        device memory above the reserve, and trains it on train_frames (a
        device uint8 tensor [N, H, W, 3]).  Returns None when refused.  A
        camera admitted after start() joins the running server between two
        of its steps."""
        torch = self.torch
        cam = Camera(-1, width, height, K, dtype)
        need = cog.cog_state_bytes(cam.params) + 2 * cam.P * 4 + (1 << 20)
        free, _ = torch.cuda.mem_get_info(self.dev)
        if free - need < self.reserve:
            self.refused.append((width, height, K, dtype, need))
            return None
        stream = torch.cuda.current_stream(self.dev)
        cam.ctx = cog.cog_create(cam.params, stream.cuda_stream)
        cog.cog_train_prior(cam.ctx, train_frames, train_frames.shape[0])
        cog.cog_sync(cam.ctx)
        if not self.keep_masks:
            cam.mask_ring = [self.mask_arena.take((height, width)) for _ in range(self.RING)]
        if self.srv is not None:
            try:
                idx = cog.cog_server_add(self.srv, cam.ctx)
            except cog.CogError:
                cog.cog_destroy(cam.ctx)
                self.refused.append((width, height, K, dtype, need))
                return None
            # the lowest index a camera has left, else the next one
            free = [i for i, c in enumerate(self.cameras) if c is None]
            assert idx == (free[0] if free else len(self.cameras))
            cam.id = idx
            if idx == len(self.cameras):
                self.cameras.append(cam)
            else:
                self.cameras[idx] = cam
            return cam
        cam.id = len(self.cameras)
        self.cameras.append(cam)
        return cam

    def leave(self, cam: Camera) -> None:
        """cam leaves the running server once its submitted frames are done;
        its model and buffers are freed and its index goes to the next
        admission."""
        assert self.srv is not None and self.cameras[cam.id] is cam
        ctx = cog.cog_server_remove(self.srv, cam.id)
        cog.cog_destroy(ctx)
        cam.ctx = None
        self.cameras[cam.id] = None
        self.results.pop(cam.id, None)   # its masks stay in cam.masks

    def start(self, warmup_frames=None):
        """Hands the admitted cameras to the native server and starts it.
        warmup_frames (optional): camera id -> list of host frames, served
        first and left out of the statistics; they take each camera's first
        steps (slot buffers, the batch graph's first launch)."""
        assert all(c is not None for c in self.cameras)
        self.srv = cog.cog_server_create([c.ctx for c in self.cameras])
        if warmup_frames:
            for cam in self.cameras:
                for f in warmup_frames.get(cam.id, []):
                    self.submit(cam, f)
            cog.cog_server_drain(self.srv, 120000)
            cog.cog_server_reset_stats(self.srv)

    def submit(self, cam: Camera, frame_host, t_arrival: float | None = None):
        """Queues a host frame (pinned uint8 tensor [H, W, 3], alive until
        the frame is done) for cam.  t_arrival is accepted for interface
        compatibility; latency is measured from this call."""
        if self.keep_masks:
            mask = np.empty((cam.height, cam.width), np.uint8)
            self.results[cam.id].append((cam.seq, mask))
            cam.masks.append((cam.seq, mask))
            self._keep.append(frame_host)
        else:
            mask = cam.mask_ring[cam.seq % self.RING]
        cam.seq += 1
        cog.cog_server_submit(self.srv, cam.id, frame_host, mask)

    def stop(self, timeout_ms: int = 120000):
        """Waits until every submitted frame is done and returns the serving
        statistics."""
        cog.cog_server_drain(self.srv, timeout_ms)
        st = cog.cog_server_read_stats(self.srv)
        self.timeline = cog.cog_server_read_timeline(self.srv)
        self.steps = cog.cog_server_read_steps(self.srv)
        self._keep = []
        wall = st["wall_s"]
        return {"frames": st["frames"], "steps": st["steps"], "wall_s": round(wall, 3),
                "mpixel_per_s": round(st["pixels"] / wall / 1e6, 1) if wall > 0 else 0.0,
                "latency_ms": {"p50": round(st["p50_ms"], 3) if st["frames"] else None,
                               "p99": round(st["p99_ms"], 3) if st["frames"] else None,
                               "max": round(st["max_ms"], 3) if st["frames"] else None},
                # where the latency goes: waiting for the worker to take the
                # frame, the frame's service (upload, step, download), and
                # the host time the worker needed to issue a step
                "latency_split_ms": {"wait_p50": round(st["wait_p50_ms"], 3), "wait_p99": round(st["wait_p99_ms"], 3),
                                     "service_p50": round(st["service_p50_ms"], 3),
                                     "service_p99": round(st["service_p99_ms"], 3),
                                     "enqueue_p99": round(st["enqueue_p99_ms"], 3),
                                     "enqueue_max": round(st["enqueue_max_ms"], 3)},
                "cameras": sum(c is not None for c in self.cameras), "refused": len(self.refused)}

    def close(self):
        if self.srv is not None:
            cog.cog_server_destroy(self.srv)
            self.srv = None
        for c in self.cameras:
            if c is not None:
                cog.cog_destroy(c.ctx)
                c.mask_ring = []
        self.cameras = []
        self.arena.release()
        self.mask_arena.release()
