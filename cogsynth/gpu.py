"""CUDA twin of ``cogsynth.scene``: renders whole workloads on the device.

The static scene maps and the per-frame descriptors come from the numpy
``Scene`` (host); the device kernel only evaluates the per-pixel recipe, so
its frames are bit-identical to ``Scene.render``.  Input generation only.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

from .scene import MAX_OBJ, Scene

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc", "synth.cu")
_LIB = os.path.join(_HERE, "libcogsynth.so")
_lock = threading.Lock()
_lib = None

FRAME_DT = np.dtype([("noise_base", "<u8"), ("offset", "<i4"), ("sway", "<i4"), ("n_obj", "<i4"),
                     ("pad", "<i4"), ("modes", "<u4", (8,)), ("obj", "<i4", (MAX_OBJ, 8))])
assert FRAME_DT.itemsize == 568


class _SceneC(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("n_blobs", C.c_int32), ("pad", C.c_int32),
                ("sway_x0", C.c_int32), ("sway_y0", C.c_int32), ("sway_x1", C.c_int32),
                ("sway_y1", C.c_int32), ("bg", C.c_void_p), ("sig16", C.c_void_p),
                ("blob_id", C.c_void_p), ("blob_delta", C.c_void_p)]


def build_synth(force: bool = False) -> str:
    hdr = os.path.join(_HERE, "csrc", "cogsynth.h")
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
            os.path.getmtime(_SRC), os.path.getmtime(hdr)):
        return _LIB
    nvcc = "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc"
    cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-Xcompiler", "-fPIC",
           "-shared", "-cudart", "static", "-o", _LIB + ".tmp", _SRC]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {_SRC}:\n{r.stdout}\n{r.stderr}")
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB):
                raise ImportError("libcogsynth.so is not built; run __graft_entry__.build()")
            lib = C.CDLL(_LIB)
            lib.cogsynth_render.argtypes = [C.POINTER(_SceneC), C.c_void_p, C.c_int32, C.c_void_p,
                                            C.c_void_p, C.c_void_p]
            lib.cogsynth_render.restype = C.c_int
            _lib = lib
    return _lib


def frame_descs(scene: Scene, t0: int, n: int) -> np.ndarray:
    out = np.zeros(n, FRAME_DT)
    for i in range(n):
        d = scene.frame_desc(t0 + i)
        out[i]["noise_base"] = d["noise_base"]
        out[i]["offset"] = d["offset"]
        out[i]["sway"] = d["sway"]
        objs = d["objects"]
        out[i]["n_obj"] = len(objs)
        for j, o in enumerate(objs):
            out[i]["obj"][j] = o
        m = d["modes"]
        words = np.zeros(8, np.uint32)
        for b in np.nonzero(m)[0]:
            words[b >> 5] |= np.uint32(1 << (b & 31))
        out[i]["modes"] = words
    return out


class GpuScene:
    """Device copy of a scene's static maps; renders frames into torch tensors."""

    def __init__(self, scene: Scene, device="cuda"):
        import torch
        self.torch = torch
        self.scene = scene
        self.device = torch.device(device)
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(self.device)  # noqa: E731
        self.bg = t(scene.bg.astype(np.uint8))
        self.sig16 = t(scene.sig16.astype(np.uint8))
        self.blob_id = t(scene.blob_id.astype(np.int16))
        delta = scene.blob_delta if len(scene.blob_delta) else np.zeros((1, 3), np.int16)
        self.blob_delta = t(delta.astype(np.int16))
        x0, y0, x1, y1 = scene.sway_rect
        self.c = _SceneC(scene.width, scene.height, len(scene.blob_delta), 0, x0, y0, x1, y1,
                         self.bg.data_ptr(), self.sig16.data_ptr(), self.blob_id.data_ptr(),
                         self.blob_delta.data_ptr())

    def render(self, t0: int, n: int, out=None, gt: bool = False, chunk: int = 256):
        """Frames t0..t0+n-1 as a uint8 tensor [n, H, W, 3] (and [n, H, W] truth)."""
        torch = self.torch
        sc = self.scene
        if out is None:
            out = torch.empty((n, sc.height, sc.width, 3), dtype=torch.uint8, device=self.device)
        g = torch.empty((n, sc.height, sc.width), dtype=torch.uint8, device=self.device) if gt else None
        lib = _load()
        stream = torch.cuda.current_stream(self.device).cuda_stream
        for s in range(0, n, chunk):
            m = min(chunk, n - s)
            d = torch.from_numpy(frame_descs(sc, t0 + s, m).view(np.uint8)).to(self.device)
            r = lib.cogsynth_render(C.byref(self.c), d.data_ptr(), m, out[s:s + m].data_ptr(),
                                    g[s:s + m].data_ptr() if gt else None, stream)
            if r != 0:
                raise RuntimeError(f"cogsynth_render failed with CUDA error {r}")
            torch.cuda.current_stream(self.device).synchronize()   # descriptors are freed next
        return (out, g) if gt else out
