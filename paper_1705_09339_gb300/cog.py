"""Thin ctypes binding of libcog.so (include/cog.h), same names as the C ABI.

This module only marshals arguments: every step of the method runs in the
CUDA library.  Device buffers are passed as torch CUDA tensors (their
``data_ptr()``); PyTorch supplies device memory and streams only.  There is
no CPU fallback: if the library is missing or fails to load, importing this
module raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# COG_LIB_VARIANT=debug loads the COG_DEBUG build (libcog_debug.so, every
# data-dependent kernel index bounds-checked) instead of libcog.so
LIB_PATH = os.path.join(_PKG, "libcog_debug.so" if os.environ.get("COG_LIB_VARIANT") == "debug" else "libcog.so")

COG_OK, COG_ERR_INVALID_ARG, COG_ERR_OOM, COG_ERR_CUDA, COG_ERR_STATE, COG_ERR_TIMEOUT, COG_ERR_DEVICE = range(7)
STATUS_NAMES = ["COG_OK", "COG_ERR_INVALID_ARG", "COG_ERR_OOM", "COG_ERR_CUDA", "COG_ERR_STATE",
                "COG_ERR_TIMEOUT", "COG_ERR_DEVICE"]
COG_F32, COG_F16, COG_BF16 = 0, 1, 2
COG_FD, COG_RGA, COG_CONF, COG_ILLUM, COG_SAMPLE, COG_MODE1, COG_PERCHAN = 1, 2, 4, 8, 16, 32, 64
COG_ALL = 15
DTYPES = {"f32": COG_F32, "f16": COG_F16, "bf16": COG_BF16}


class cog_params(C.Structure):
    _fields_ = [
        ("width", C.c_int32), ("height", C.c_int32), ("K", C.c_int32), ("state_dtype", C.c_int32),
        ("alpha", C.c_float), ("lambda_", C.c_float), ("T_bg", C.c_float), ("w_init", C.c_float),
        ("var_init", C.c_float), ("var_min", C.c_float), ("var_max", C.c_float), ("tau_fd", C.c_float),
        ("eta_conf", C.c_float), ("c_halt", C.c_float), ("w_illum", C.c_float),
        ("q_null", C.c_int32), ("kde_bw", C.c_int32), ("r1", C.c_int32), ("r2", C.c_int32),
        ("illum_permille", C.c_int32), ("flags", C.c_uint32), ("c_skip", C.c_float),
        ("skip_period", C.c_int32), ("kde_bits", C.c_int32),
    ]


class cog_stats(C.Structure):
    _fields_ = [("n_stage", C.c_int64 * 6), ("n_gmm", C.c_int64), ("illum_flag", C.c_int32),
                ("frame", C.c_int32)]

    def as_dict(self) -> dict:
        return dict(n_stage=list(self.n_stage), n_gmm=int(self.n_gmm), illum_flag=int(self.illum_flag),
                    frame=int(self.frame))


class cog_group_stats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("converged", C.c_int32), ("n", C.c_int64 * 3),
                ("n_core", C.c_int64 * 3), ("code_sum", (C.c_int64 * 2) * 3), ("code_sq_sum", (C.c_int64 * 2) * 3),
                ("centroid", (C.c_double * 2) * 3), ("sd", (C.c_double * 2) * 3), ("w1", C.c_double * 3),
                ("mu1", (C.c_double * 3) * 3), ("v1", C.c_double * 3)]

    def as_dict(self) -> dict:
        def conv(x):
            return [conv(v) for v in x] if isinstance(x, C.Array) else x
        return {n: conv(getattr(self, n)) for n, _ in self._fields_}


class cog_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("frames", C.c_int64), ("steps", C.c_int64), ("pixels", C.c_int64),
                ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("max_ms", C.c_double), ("wall_s", C.c_double),
                ("wait_p50_ms", C.c_double), ("wait_p99_ms", C.c_double), ("service_p50_ms", C.c_double),
                ("service_p99_ms", C.c_double), ("enqueue_p99_ms", C.c_double), ("enqueue_max_ms", C.c_double)]

    def as_dict(self) -> dict:
        return {n: getattr(self, n) for n, _ in self._fields_}


class cog_layout(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ("total", "ctl", "jl", "conf", "s1", "s1_bytes", "gmm", "rec_bytes",
                                          "queue", "kde", "elem_bytes", "kde_row")]


class CogError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 7 else status}: {msg}")
        self.status = status


def _load() -> C.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{os.path.basename(LIB_PATH)} is not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = C.CDLL(LIB_PATH)
    vp, i32, sz = C.c_void_p, C.c_int32, C.c_size_t
    P = C.POINTER
    sig = {
        "cog_default_params": (None, [P(cog_params), i32, i32, i32]),
        "cog_state_bytes": (C.c_int, [P(cog_params), P(sz)]),
        "cog_state_layout": (C.c_int, [P(cog_params), P(cog_layout)]),
        "cog_create": (C.c_int, [P(cog_params), vp, vp, P(vp)]),
        "cog_train_prior": (C.c_int, [vp, vp, i32]),
        "cog_apply": (C.c_int, [vp, vp, vp, vp, P(cog_stats)]),
        "cog_apply_clip": (C.c_int, [vp, vp, i32, vp, vp, P(cog_stats)]),
        "cog_clip_runs": (C.c_int, [vp, P(i32)]),
        "cog_selftest_bounded_wait": (C.c_int, [i32, P(C.c_uint32), P(C.c_double)]),
        "cog_probe_stream": (C.c_int, [vp, vp, vp, vp, vp, vp, C.c_int64, vp]),
        "cog_group": (C.c_int, [vp, vp, i32, vp, vp, P(cog_group_stats)]),
        "cog_group_cluster": (C.c_int, [vp, vp, i32, vp, P(cog_group_stats)]),
        "cog_apply_plain_gmm": (C.c_int, [vp, vp, vp]),
        "cog_apply_host": (C.c_int, [vp, vp, vp]),
        "cog_apply_host_noalloc": (C.c_int, [vp, vp, vp]),
        "cog_apply_host_frames": (C.c_int, [vp, vp, i32, vp]),
        "cog_read_stats": (C.c_int, [vp, P(cog_stats), P(cog_stats)]),
        "cog_sync": (C.c_int, [vp]),
        "cog_debug_build": (C.c_int32, []),
        "cog_export_state": (C.c_int, [vp, vp, sz]),
        "cog_import_state": (C.c_int, [vp, vp, sz]),
        "cog_info": (C.c_int, [vp, P(C.c_int64), P(vp)]),
        "cog_profile_begin": (C.c_int, [vp, i32]),
        "cog_set_launch": (C.c_int, [vp, i32, i32, i32]),
        "cog_set_l2_fetch_bytes": (C.c_int, [i32]),
        "cog_host_alloc": (C.c_int, [sz, P(vp)]),
        "cog_host_free": (C.c_int, [vp]),
        "cog_profile_end": (C.c_int, [vp, P(C.c_double), P(C.c_double), P(C.c_int64)]),
        "cog_last_error_string": (C.c_char_p, [vp]),
        "cog_destroy": (C.c_int, [vp]),
        "cog_batch_create": (C.c_int, [P(vp), i32, vp, P(vp)]),
        "cog_batch_apply": (C.c_int, [vp, P(vp), P(vp)]),
        "cog_batch_apply_active": (C.c_int, [vp, P(vp), P(vp), vp]),
        "cog_batch_sync": (C.c_int, [vp]),
        "cog_batch_last_error_string": (C.c_char_p, [vp]),
        "cog_batch_destroy": (C.c_int, [vp]),
        "cog_server_create": (C.c_int, [P(vp), i32, P(vp)]),
        "cog_server_submit": (C.c_int, [vp, i32, vp, vp]),
        "cog_server_add": (C.c_int, [vp, vp, P(i32)]),
        "cog_server_remove": (C.c_int, [vp, i32, P(vp)]),
        "cog_server_drain": (C.c_int, [vp, i32]),
        "cog_server_read_stats": (C.c_int, [vp, P(cog_server_stats)]),
        "cog_server_read_latencies": (C.c_int, [vp, vp, vp, C.c_int64, P(C.c_int64)]),
        "cog_server_read_timeline": (C.c_int, [vp, vp, vp, vp, C.c_int64, P(C.c_int64)]),
        "cog_server_read_steps": (C.c_int, [vp, vp, vp, C.c_int64, P(C.c_int64)]),
        "cog_server_reset_stats": (C.c_int, [vp]),
        "cog_server_last_error_string": (C.c_char_p, [vp]),
        "cog_server_destroy": (C.c_int, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def _check(status: int, ctx=None):
    if status != COG_OK:
        msg = lib.cog_last_error_string(ctx)
        raise CogError(status, msg.decode() if msg else "")


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def cog_default_params(width: int, height: int, K: int = 3, **over) -> cog_params:
    p = cog_params()
    lib.cog_default_params(C.byref(p), width, height, K)
    for k, v in over.items():
        if k == "state_dtype" and isinstance(v, str):
            v = DTYPES[v]
        setattr(p, "lambda_" if k == "lambda" else k, v)
    return p


def cog_state_layout(p: cog_params) -> cog_layout:
    l = cog_layout()
    _check(lib.cog_state_layout(C.byref(p), C.byref(l)))
    return l


def cog_state_bytes(p: cog_params) -> int:
    n = C.c_size_t()
    _check(lib.cog_state_bytes(C.byref(p), C.byref(n)))
    return n.value


def cog_create(p: cog_params, stream: int | None = None, state=None) -> C.c_void_p:
    ctx = C.c_void_p()
    _check(lib.cog_create(C.byref(p), stream, _ptr(state), C.byref(ctx)))
    return ctx


def cog_train_prior(ctx, frames, n_frames: int) -> None:
    _check(lib.cog_train_prior(ctx, _ptr(frames), n_frames), ctx)


def cog_apply(ctx, frame, mask, stagemap=None, want_stats: bool = False):
    st = cog_stats() if want_stats else None
    _check(lib.cog_apply(ctx, _ptr(frame), _ptr(mask), _ptr(stagemap), C.byref(st) if st else None), ctx)
    return st.as_dict() if st else None


def cog_apply_clip(ctx, frames, n_frames: int, masks, stagemaps=None, want_stats: bool = False):
    """n_frames consecutive frames ([n, H, W, 3] bytes) through the cascade;
    identical to n_frames cog_apply calls.  Returns per-frame stats dicts
    when asked."""
    st = (cog_stats * n_frames)() if want_stats else None
    _check(lib.cog_apply_clip(ctx, _ptr(frames), int(n_frames), _ptr(masks), _ptr(stagemaps), st), ctx)
    return [s.as_dict() for s in st] if st is not None else None


def cog_clip_runs(ctx) -> int:
    r = C.c_int32(0)
    _check(lib.cog_clip_runs(ctx, C.byref(r)), ctx)
    return r.value


def cog_selftest_bounded_wait(limit_ms: int):
    """Runs the bounded grid-wide wait on a count nothing completes;
    returns (device error bits it set, kernel milliseconds)."""
    w, ms = C.c_uint32(0), C.c_double(0.0)
    _check(lib.cog_selftest_bounded_wait(int(limit_ms), C.byref(w), C.byref(ms)))
    return w.value, ms.value


def cog_group(ctx, frames, n_frames: int, codes, labels) -> dict:
    """Spatio-temporal grouping on the training frames (uint8 [N, H, W, 3]
    on the GPU): fills codes (uint16 [2, P]: code_v, code_w) and labels
    (uint8 [P]: cluster | 0x80 for a core pixel); returns the statistics."""
    st = cog_group_stats()
    _check(lib.cog_group(ctx, _ptr(frames), int(n_frames), _ptr(codes), _ptr(labels), C.byref(st)), ctx)
    return st.as_dict()


def cog_group_cluster(ctx, codes, max_steps: int, labels) -> dict:
    """Grouping steps 3-6 on given codes (uint16 [2, P] on the GPU): the
    first assignment and at most max_steps Lloyd steps, then the Eq. 3
    cores; fills labels (uint8 [P]) and returns the statistics."""
    st = cog_group_stats()
    _check(lib.cog_group_cluster(ctx, _ptr(codes), int(max_steps), _ptr(labels), C.byref(st)), ctx)
    return st.as_dict()


def cog_probe_stream(jl_in, conf_in, frame, jl_out, conf_out, mask, stream=None) -> None:
    """Streaming probe over stage 0's planes (no arithmetic): jl_out = this
    frame with jl_in's labels, conf_out = conf_in, mask = jl_in's labels.
    jl: uint32 [P], conf: 16-bit [P], frame: uint8 [P, 3], mask: uint8 [P]."""
    P = int(mask.numel())
    _check(lib.cog_probe_stream(_ptr(jl_in), _ptr(conf_in), _ptr(frame), _ptr(jl_out), _ptr(conf_out),
                                _ptr(mask), P, stream))


def cog_apply_plain_gmm(ctx, frame, mask) -> None:
    _check(lib.cog_apply_plain_gmm(ctx, _ptr(frame), _ptr(mask)), ctx)


def cog_apply_host(ctx, frame: np.ndarray, mask: np.ndarray) -> None:
    assert frame.dtype == np.uint8 and mask.dtype == np.uint8
    assert frame.flags.c_contiguous and mask.flags.c_contiguous
    _check(lib.cog_apply_host(ctx, frame.ctypes.data, mask.ctypes.data), ctx)


def cog_apply_host_frames(ctx, frames: np.ndarray, masks: np.ndarray) -> None:
    """frames [n, H, W, 3] and masks [n, H, W] in host memory (pinned for
    overlap); copies pipelined with the kernels."""
    assert frames.dtype == np.uint8 and masks.dtype == np.uint8
    assert frames.flags.c_contiguous and masks.flags.c_contiguous and frames.shape[0] == masks.shape[0]
    _check(lib.cog_apply_host_frames(ctx, frames.ctypes.data, int(frames.shape[0]), masks.ctypes.data), ctx)


def cog_apply_host_noalloc(ctx, frame: np.ndarray, mask: np.ndarray) -> None:
    """cog_apply_host staged through the library's static device array
    (no device allocation; frames up to 1920 x 1080)."""
    assert frame.dtype == np.uint8 and mask.dtype == np.uint8
    assert frame.flags.c_contiguous and mask.flags.c_contiguous
    _check(lib.cog_apply_host_noalloc(ctx, frame.ctypes.data, mask.ctypes.data), ctx)


def cog_read_stats(ctx):
    a, b = cog_stats(), cog_stats()
    _check(lib.cog_read_stats(ctx, C.byref(a), C.byref(b)), ctx)
    return a.as_dict(), b.as_dict()


def cog_sync(ctx) -> None:
    _check(lib.cog_sync(ctx), ctx)


def cog_export_state(ctx, p: cog_params) -> np.ndarray:
    n = cog_state_layout(p).total
    buf = np.empty(n, np.uint8)
    _check(lib.cog_export_state(ctx, buf.ctypes.data, n), ctx)
    return buf


def cog_import_state(ctx, buf: np.ndarray) -> None:
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    _check(lib.cog_import_state(ctx, buf.ctypes.data, buf.size), ctx)


def cog_info(ctx):
    n, s = C.c_int64(), C.c_void_p()
    _check(lib.cog_info(ctx, C.byref(n), C.byref(s)), ctx)
    return n.value, s.value


def cog_set_l2_fetch_bytes(nbytes: int) -> None:
    _check(lib.cog_set_l2_fetch_bytes(nbytes))


def cog_set_launch(ctx, k1_threads: int = 128, k2_threads: int = 64, k2_ctas_per_sm: int = 0) -> None:
    _check(lib.cog_set_launch(ctx, k1_threads, k2_threads, k2_ctas_per_sm), ctx)


def cog_profile_begin(ctx, max_frames: int) -> None:
    _check(lib.cog_profile_begin(ctx, max_frames), ctx)


def cog_profile_end(ctx):
    """Returns (stage01_ms, stage2_ms, frames) summed over the recorded frames."""
    a, b, n = C.c_double(), C.c_double(), C.c_int64()
    _check(lib.cog_profile_end(ctx, C.byref(a), C.byref(b), C.byref(n)), ctx)
    return a.value, b.value, n.value


def cog_last_error_string(ctx=None) -> str:
    m = lib.cog_last_error_string(ctx)
    return m.decode() if m else ""


def cog_destroy(ctx) -> None:
    _check(lib.cog_destroy(ctx))


def _bcheck(status: int, b=None):
    if status != COG_OK:
        msg = lib.cog_batch_last_error_string(b)
        raise CogError(status, msg.decode() if msg else "")


def cog_batch_create(ctxs, stream: int):
    arr = (C.c_void_p * len(ctxs))(*[c.value if isinstance(c, C.c_void_p) else c for c in ctxs])
    b = C.c_void_p()
    _bcheck(lib.cog_batch_create(arr, len(ctxs), stream, C.byref(b)))
    return b


def cog_batch_apply(b, frames, masks) -> None:
    n = len(frames)
    fa = (C.c_void_p * n)(*[_ptr(f) for f in frames])
    ma = (C.c_void_p * n)(*[_ptr(m) for m in masks])
    _bcheck(lib.cog_batch_apply(b, fa, ma), b)


def cog_batch_apply_active(b, frames, masks, active) -> None:
    """active: sequence of n truthy flags; frames/masks of inactive streams
    may be None."""
    n = len(frames)
    fa = (C.c_void_p * n)(*[_ptr(f) for f in frames])
    ma = (C.c_void_p * n)(*[_ptr(m) for m in masks])
    act = np.ascontiguousarray(np.asarray(active, dtype=np.uint8))
    _bcheck(lib.cog_batch_apply_active(b, fa, ma, act.ctypes.data), b)


def cog_batch_sync(b) -> None:
    _bcheck(lib.cog_batch_sync(b), b)


def cog_batch_destroy(b) -> None:
    _bcheck(lib.cog_batch_destroy(b))


# ----------------------------------------------------------------------------
# Decoding an exported state image into numpy views (documented layout).
# ----------------------------------------------------------------------------
_NP_DT = {COG_F32: np.float32, COG_F16: np.float16}


def _plane(buf: np.ndarray, off: int, n: int, dtype) -> np.ndarray:
    itemsize = np.dtype(dtype).itemsize
    return buf[off:off + n * itemsize].view(dtype)


def _bf16_to_f32(u16: np.ndarray) -> np.ndarray:
    return (u16.astype(np.uint32) << 16).view(np.float32)


def _s1_view(buf, L, P, p):
    """Stage-1 records as (values [P, 6] float64, qab [P] uint16, top [P]
    uint8: the mixture component the record mirrors under COG_MODE1)."""
    rb = int(L.s1_bytes)
    raw = buf[L.s1:L.s1 + P * rb].reshape(P, rb)
    if p.state_dtype == COG_F32:
        vals = raw[:, :24].copy().view(np.float32).astype(np.float64)
        qab = raw[:, 24:28].copy().view(np.uint32).reshape(P).astype(np.uint16)
        top = raw[:, 28].copy()
    else:
        h = raw[:, :12].copy().view(np.uint16)
        vals = (_bf16_to_f32(h) if p.state_dtype == COG_BF16 else h.view(np.float16)).astype(np.float64)
        qab = raw[:, 12:14].copy().view(np.uint16).reshape(P)
        top = raw[:, 14].copy()
    return vals.reshape(P, 6), qab, top


def _prior_levels(rows: np.ndarray) -> np.ndarray:
    """Prior rows [P, 3, kde_row] -> one level per grey value [P, 3, 256]
    (4-bit rows hold level 2j in the low and 2j+1 in the high nibble of
    byte j)."""
    if rows.shape[2] == 256:
        return rows
    q = np.empty(rows.shape[:2] + (256,), np.uint8)
    q[:, :, 0::2] = rows & 0xF
    q[:, :, 1::2] = rows >> 4
    return q


def decode_state(buf: np.ndarray, p: cog_params) -> dict:
    """FP64 copies of the model planes of an exported state image:
    w [P,K], mu [P,K,3], var [P,K,3], rga_m [P,3], rga_v [P,3], conf [P],
    label [P], prev [P,3], kde [P,3,256] (levels of 255, or of 15 with
    kde_bits = 4), qa [P], qb [P], top [P]; with
    COG_PERCHAN the weights are per channel: wc [P,3,K] instead of w."""
    L = cog_state_layout(p)
    P, K = p.width * p.height, p.K
    Pp = (P + 4095) // 4096 * 4096

    def vals(off, n):
        if p.state_dtype == COG_BF16:
            return _bf16_to_f32(_plane(buf, off, n, np.uint16)).astype(np.float64)
        return _plane(buf, off, n, _NP_DT[p.state_dtype]).astype(np.float64)

    jl = _plane(buf, L.jl, P, np.uint32)
    prev = np.stack([(jl >> (8 * c)) & 0xFF for c in range(3)], axis=1).astype(np.uint8)
    label = (jl >> 24).astype(np.uint8)
    conf = vals(L.conf, P)
    s1, qab, top = _s1_view(buf, L, P, p)
    rec_elems = L.rec_bytes // L.elem_bytes
    if p.state_dtype == COG_BF16:
        recs = _bf16_to_f32(_plane(buf, L.gmm, Pp * rec_elems, np.uint16)).astype(np.float64)
    else:
        recs = _plane(buf, L.gmm, Pp * rec_elems, _NP_DT[p.state_dtype]).astype(np.float64)
    kde = _prior_levels(buf[L.kde:L.kde + P * 3 * L.kde_row].reshape(P, 3, L.kde_row))
    out = dict(rga_m=s1[:, :3].copy(), rga_v=s1[:, 3:].copy(), conf=conf, label=label, prev=prev,
               kde=kde, qa=(qab & 0xFF).astype(np.uint8), qb=(qab >> 8).astype(np.uint8), top=top)
    if p.flags & COG_PERCHAN:
        # per component (w0 w1 w2 mu0 mu1 mu2 v0 v1 v2); wc [P, 3, K]
        recs = recs.reshape(Pp, rec_elems)[:P, :9 * K].reshape(P, K, 9)
        out.update(wc=recs[:, :, 0:3].transpose(0, 2, 1).copy(), mu=recs[:, :, 3:6].copy(),
                   var=recs[:, :, 6:9].copy())
    else:
        recs = recs.reshape(Pp, rec_elems)[:P, :7 * K].reshape(P, K, 7)
        out.update(w=recs[:, :, 0].copy(), mu=recs[:, :, 1:4].copy(), var=recs[:, :, 4:7].copy())
    return out


def _to_storage(arr, dtype) -> np.ndarray:
    """float64 values -> raw little-endian storage words (uint16/float32)."""
    arr = np.asarray(arr, np.float64)
    if dtype == COG_BF16:
        f = arr.astype(np.float32).view(np.uint32)
        return ((f + 0x7FFF + ((f >> 16) & 1)) >> 16).astype(np.uint16)
    return arr.astype(_NP_DT[dtype])


def encode_state(buf: np.ndarray, p: cog_params, st: dict) -> np.ndarray:
    """Writes model planes (same keys as decode_state) into a state image.
    Used to start the CUDA path and the oracle from one seeded state."""
    L = cog_state_layout(p)
    P, K = p.width * p.height, p.K
    Pp = (P + 4095) // 4096 * 4096
    out = buf.copy()
    jl = (st["prev"][:, 0].astype(np.uint32) | (st["prev"][:, 1].astype(np.uint32) << 8)
          | (st["prev"][:, 2].astype(np.uint32) << 16) | (st["label"].astype(np.uint32) << 24))
    out[L.jl:L.jl + 4 * P] = jl.view(np.uint8)
    c = _to_storage(st["conf"], p.state_dtype)
    out[L.conf:L.conf + c.nbytes] = c.view(np.uint8)
    rb = int(L.s1_bytes)
    rec = np.zeros((P, rb), np.uint8)
    v = _to_storage(np.concatenate([st["rga_m"], st["rga_v"]], axis=1), p.state_dtype).reshape(P, 6)
    rec[:, :v.itemsize * 6] = v.view(np.uint8).reshape(P, -1)
    qab = st["qa"].astype(np.uint32) | (st["qb"].astype(np.uint32) << 8)
    top = np.asarray(st.get("top", np.zeros(P)), np.uint8)
    if p.state_dtype == COG_F32:
        rec[:, 24:28] = qab.astype(np.uint32).view(np.uint8).reshape(P, 4)
        rec[:, 28] = top
    else:
        rec[:, 12:14] = qab.astype(np.uint16).view(np.uint8).reshape(P, 2)
        rec[:, 14] = top
    out[L.s1:L.s1 + P * rb] = rec.reshape(-1)
    rec_elems = L.rec_bytes // L.elem_bytes
    recs = np.zeros((Pp, rec_elems))
    if p.flags & COG_PERCHAN:
        r = np.concatenate([st["wc"].transpose(0, 2, 1), st["mu"], st["var"]], axis=2).reshape(P, 9 * K)
        recs[:P, :9 * K] = r
    else:
        r = np.concatenate([st["w"][:, :, None], st["mu"], st["var"]], axis=2).reshape(P, 7 * K)
        recs[:P, :7 * K] = r
    g = _to_storage(recs, p.state_dtype)
    out[L.gmm:L.gmm + g.nbytes] = g.view(np.uint8).reshape(-1)
    q = np.asarray(st["kde"], np.uint8).reshape(P, 3, 256)
    if L.kde_row == 128:
        q = (q[:, :, 0::2] & 0xF) | ((q[:, :, 1::2] & 0xF) << 4)
    out[L.kde:L.kde + P * 3 * L.kde_row] = q.reshape(-1)
    return out


# ----------------------------------------------------------------------------
# Native frame server (continuous batching of many camera streams).
# ----------------------------------------------------------------------------
def _scheck(status: int, srv=None):
    if status != COG_OK:
        msg = lib.cog_server_last_error_string(srv)
        raise CogError(status, msg.decode() if msg else "")


def cog_host_alloc(nbytes: int) -> int:
    """Page-locked host memory (cog_host_alloc); returns its address."""
    p = C.c_void_p()
    _check(lib.cog_host_alloc(int(nbytes), C.byref(p)))
    return p.value


def cog_host_free(ptr: int) -> None:
    _check(lib.cog_host_free(ptr))


def cog_server_create(ctxs) -> C.c_void_p:
    arr = (C.c_void_p * len(ctxs))(*[c.value if isinstance(c, C.c_void_p) else c for c in ctxs])
    srv = C.c_void_p()
    _scheck(lib.cog_server_create(arr, len(ctxs), C.byref(srv)))
    return srv


def cog_server_add(srv, ctx) -> int:
    """A further trained context joins the running server; returns its
    stream index."""
    idx = C.c_int32(-1)
    _scheck(lib.cog_server_add(srv, ctx, C.byref(idx)), srv)
    return idx.value


def cog_server_remove(srv, stream: int) -> C.c_void_p:
    """Camera `stream` leaves the running server once its submitted frames
    are done; returns its context, which belongs to the caller again."""
    ctx = C.c_void_p()
    _scheck(lib.cog_server_remove(srv, int(stream), C.byref(ctx)), srv)
    return ctx


def cog_server_submit(srv, stream: int, frame_host, mask_host) -> None:
    """frame_host / mask_host: host tensors or numpy arrays (page-locked for
    overlap) that stay alive until the frame is done."""
    _scheck(lib.cog_server_submit(srv, int(stream), _host_ptr(frame_host), _host_ptr(mask_host)), srv)


def cog_server_drain(srv, timeout_ms: int = 60000) -> None:
    _scheck(lib.cog_server_drain(srv, int(timeout_ms)), srv)


def cog_server_read_stats(srv) -> dict:
    st = cog_server_stats()
    _scheck(lib.cog_server_read_stats(srv, C.byref(st)), srv)
    return st.as_dict()


def cog_server_read_latencies(srv):
    """(submission ms, latency ms) arrays of the frames done, in completion order."""
    n = C.c_int64(0)
    _scheck(lib.cog_server_read_latencies(srv, None, None, 0, C.byref(n)), srv)
    t = np.empty(n.value, np.float32)
    lat = np.empty(n.value, np.float32)
    _scheck(lib.cog_server_read_latencies(srv, t.ctypes.data, lat.ctypes.data, n.value, C.byref(n)), srv)
    return t, lat


def cog_server_read_timeline(srv):
    """(submission ms, wait ms, latency ms) arrays of the frames done, in
    completion order; wait = submission until the worker took the frame."""
    n = C.c_int64(0)
    _scheck(lib.cog_server_read_timeline(srv, None, None, None, 0, C.byref(n)), srv)
    t, w, lat = (np.empty(n.value, np.float32) for _ in range(3))
    _scheck(lib.cog_server_read_timeline(srv, t.ctypes.data, w.ctypes.data, lat.ctypes.data, n.value, C.byref(n)),
            srv)
    return t, w, lat


def cog_server_read_steps(srv):
    """(enqueue ms [steps], parts [steps, 10]) of the completed steps: host
    time per step; its split into uploads, batched step, downloads (ms);
    then the GPU times of uploads, compute wait, batched step, download
    wait, downloads (ms); then the step's frames and uploaded megabytes."""
    n = C.c_int64(0)
    _scheck(lib.cog_server_read_steps(srv, None, None, 0, C.byref(n)), srv)
    e = np.empty(n.value, np.float32)
    parts = np.empty((n.value, 10), np.float32)
    _scheck(lib.cog_server_read_steps(srv, e.ctypes.data, parts.ctypes.data, n.value, C.byref(n)), srv)
    return e, parts


def cog_server_reset_stats(srv) -> None:
    _scheck(lib.cog_server_reset_stats(srv), srv)


def cog_server_destroy(srv) -> None:
    _scheck(lib.cog_server_destroy(srv))


def _host_ptr(x) -> int:
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()
