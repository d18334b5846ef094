"""ctypes wrapper of the FP64 oracle library (``libcog_oracle.so``).

Test infrastructure only.  The wrapper marshals numpy arrays; every step of
the method runs in ``cog_oracle.c``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cog_oracle.c")
_LIB = os.path.join(_HERE, "libcog_oracle.so")

ORC_FD, ORC_RGA, ORC_CONF, ORC_ILLUM, ORC_SAMPLE, ORC_MODE1, ORC_PERCHAN = 1, 2, 4, 8, 16, 32, 64
NEAR_BITS = {"fd": 1, "rga": 2, "match": 4, "bgset": 8, "rank": 16, "halt": 32, "skip": 64}

_lock = threading.Lock()
_lib = None


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP when available).  FP contraction
    is off so x86 and Arm give the same FP64 results."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "cog_oracle.h"))):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
            "-fno-fast-math", "-o", _LIB + ".tmp", _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True, text=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True, text=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _Params(C.Structure):
    _fields_ = [
        ("width", C.c_int), ("height", C.c_int), ("K", C.c_int),
        ("alpha", C.c_double), ("lambda_", C.c_double), ("T_bg", C.c_double),
        ("w_init", C.c_double), ("var_init", C.c_double), ("var_min", C.c_double),
        ("var_max", C.c_double), ("tau_fd", C.c_double), ("eta", C.c_double),
        ("c_halt", C.c_double), ("w_illum", C.c_double), ("c_skip", C.c_double),
        ("q_null", C.c_int), ("kde_bw", C.c_int), ("r1", C.c_int), ("r2", C.c_int),
        ("illum_permille", C.c_int), ("skip_period", C.c_int), ("flags", C.c_uint),
        ("kde_bits", C.c_int),
    ]


class _State(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in (
        "w", "mu", "var", "rga_m", "rga_v", "conf", "label", "prev", "kde",
        "qa", "qb", "illum", "top", "wc")]


class _Stats(C.Structure):
    _fields_ = [("n_stage", C.c_int64 * 6), ("n_gmm", C.c_int64),
                ("illum_flag", C.c_int32), ("pad", C.c_int32)]


class _GroupOut(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("converged", C.c_int32), ("n", C.c_int64 * 3),
                ("n_core", C.c_int64 * 3), ("s1", (C.c_int64 * 2) * 3), ("s2", (C.c_int64 * 2) * 3),
                ("centroid", (C.c_double * 2) * 3), ("sd", (C.c_double * 2) * 3),
                ("w1", C.c_double * 3), ("mu1", (C.c_double * 3) * 3), ("v1", C.c_double * 3),
                ("n_near", C.c_int64)]


def _group_dict(g: _GroupOut) -> dict:
    return dict(iterations=int(g.iterations), converged=int(g.converged), n=list(g.n), n_core=list(g.n_core),
                s1=[list(r) for r in g.s1], s2=[list(r) for r in g.s2],
                centroid=[list(r) for r in g.centroid], sd=[list(r) for r in g.sd],
                w1=list(g.w1), mu1=[list(r) for r in g.mu1], v1=list(g.v1), n_near=int(g.n_near))


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build_oracle()
            lib = C.CDLL(_LIB)
            lib.orc_kde_weights.argtypes = [C.c_int, C.c_void_p, C.c_int]
            lib.orc_kde_weights.restype = C.c_int
            lib.orc_train.argtypes = [C.POINTER(_Params), C.c_void_p, C.c_int, C.POINTER(_State)]
            lib.orc_train.restype = C.c_int
            lib.orc_train_near.argtypes = [C.POINTER(_Params), C.c_void_p, C.c_int, C.POINTER(_State),
                                           C.c_void_p]
            lib.orc_train_near.restype = C.c_int
            lib.orc_apply.argtypes = [C.POINTER(_Params), C.POINTER(_State), C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(_Stats)]
            lib.orc_apply.restype = C.c_int
            lib.orc_plain_gmm.argtypes = [C.POINTER(_Params)] + [C.c_void_p] * 5
            lib.orc_plain_gmm.restype = C.c_int
            lib.orc_threads.restype = C.c_int
            lib.orc_set_threads.argtypes = [C.c_int]
            lib.orc_set_threads.restype = None
            lib.orc_group_features.argtypes = [C.POINTER(_Params), C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]
            lib.orc_group_features.restype = C.c_int
            lib.orc_group_cluster.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p,
                                              C.POINTER(_GroupOut)]
            lib.orc_group_cluster.restype = C.c_int
            lib.orc_group_init.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
            lib.orc_group_init.restype = C.c_int
            lib.orc_group_centroids.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
            lib.orc_group_centroids.restype = C.c_int
            lib.orc_group_assign.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                             C.c_void_p, C.c_void_p]
            lib.orc_group_assign.restype = C.c_int64
            lib.orc_group_cores.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(_GroupOut)]
            lib.orc_group_cores.restype = C.c_int
            lib.orc_group_params.argtypes = [C.POINTER(_Params), C.POINTER(_State), C.c_void_p,
                                             C.POINTER(_GroupOut)]
            lib.orc_group_params.restype = C.c_int
            _lib = lib
    return _lib


def oracle_threads() -> int:
    return int(_load().orc_threads())


def set_threads(n: int) -> None:
    """Threads for the oracle's parallel loops (timing only)."""
    _load().orc_set_threads(int(n))


def group_cluster(code_v: np.ndarray, code_w: np.ndarray, max_iter: int = 64):
    """K-means (K = 3) over the two grouping codes and the Eq. 3 cores;
    returns (labels: cluster | 0x80 for a core pixel, result dict)."""
    cv = np.ascontiguousarray(code_v, dtype=np.uint16).ravel()
    cw = np.ascontiguousarray(code_w, dtype=np.uint16).ravel()
    assert cv.size == cw.size
    labels = np.empty(cv.size, np.uint8)
    g = _GroupOut()
    if _load().orc_group_cluster(cv.size, cv.ctypes.data, cw.ctypes.data, int(max_iter), labels.ctypes.data,
                                 C.byref(g)) != 0:
        raise ValueError("orc_group_cluster rejected its arguments")
    return labels, _group_dict(g)


def _codes(code_v, code_w):
    cv = np.ascontiguousarray(code_v, dtype=np.uint16).ravel()
    cw = np.ascontiguousarray(code_w, dtype=np.uint16).ravel()
    assert cv.size == cw.size and cv.size > 0
    return cv, cw


def group_init(code_v: np.ndarray, code_w: np.ndarray):
    """Feature scales and first centroids of the K-means: (c[3][2], sd[2])."""
    cv, cw = _codes(code_v, code_w)
    c = np.zeros((3, 2), np.float64)
    sd = np.zeros(2, np.float64)
    if _load().orc_group_init(cv.size, cv.ctypes.data, cw.ctypes.data, c.ctypes.data, sd.ctypes.data) != 0:
        raise ValueError("orc_group_init rejected its arguments")
    return c, sd


def group_centroids(code_v: np.ndarray, code_w: np.ndarray, labels: np.ndarray, c_prev: np.ndarray) -> np.ndarray:
    """One Lloyd update from the given labels (a cluster with no pixel keeps
    its centroid from c_prev)."""
    cv, cw = _codes(code_v, code_w)
    lab = np.ascontiguousarray(labels, dtype=np.uint8).ravel()
    assert lab.size == cv.size
    c = np.array(c_prev, dtype=np.float64).reshape(3, 2).copy()
    if _load().orc_group_centroids(cv.size, cv.ctypes.data, cw.ctypes.data, lab.ctypes.data, c.ctypes.data) != 0:
        raise ValueError("orc_group_centroids rejected its arguments")
    return c


def group_assign(code_v: np.ndarray, code_w: np.ndarray, c: np.ndarray, sd: np.ndarray):
    """One FP64 assignment to the centroids c; returns (labels, near)."""
    cv, cw = _codes(code_v, code_w)
    cc = np.ascontiguousarray(c, dtype=np.float64).reshape(3, 2)
    ss = np.ascontiguousarray(sd, dtype=np.float64).ravel()
    labels = np.empty(cv.size, np.uint8)
    near = np.empty(cv.size, np.uint8)
    if _load().orc_group_assign(cv.size, cv.ctypes.data, cw.ctypes.data, cc.ctypes.data, ss.ctypes.data,
                                labels.ctypes.data, near.ctypes.data) < 0:
        raise ValueError("orc_group_assign rejected its arguments")
    return labels, near.astype(bool)


def group_cores(code_v: np.ndarray, code_w: np.ndarray, labels: np.ndarray):
    """Cluster statistics and Eq. 3 cores of the given labels (core bits
    ignored); returns (labels with core bits, result dict)."""
    cv, cw = _codes(code_v, code_w)
    lab = np.array(labels, dtype=np.uint8).ravel()
    assert lab.size == cv.size
    g = _GroupOut()
    if _load().orc_group_cores(cv.size, cv.ctypes.data, cw.ctypes.data, lab.ctypes.data, C.byref(g)) != 0:
        raise ValueError("orc_group_cores rejected its arguments")
    return lab, _group_dict(g)


def default_params(width: int, height: int, K: int = 3) -> dict:
    """The oracle's own copy of the default constants (the paper states
    none; these are the readings recorded in the design notes)."""
    return dict(width=width, height=height, K=K, alpha=0.01, lambda_=2.5, T_bg=0.7,
                w_init=0.05, var_init=225.0, var_min=4.0, var_max=900.0, tau_fd=8.0,
                eta=0.125, c_halt=0.9, w_illum=0.75, c_skip=0.95, q_null=13, kde_bw=4, r1=10, r2=30,
                illum_permille=700, skip_period=4, flags=ORC_FD | ORC_RGA | ORC_CONF | ORC_ILLUM, kde_bits=8)


_OPTIONAL = {"c_skip": 0.95, "skip_period": 4, "kde_bits": 8}


def _params(p: dict) -> _Params:
    q = _Params()
    for name, _ in _Params._fields_:
        key = "lambda" if name == "lambda_" and "lambda" in p else name
        setattr(q, name, p[key] if key in p else _OPTIONAL[key])
    return q


def kde_weights(bw: int) -> np.ndarray:
    g = np.zeros(3 * bw + 1, dtype=np.int64)
    r = _load().orc_kde_weights(bw, g.ctypes.data, g.size)
    if r < 0:
        raise ValueError("bad bandwidth")
    return g


class OracleState:
    """FP64 model state of P pixels (numpy arrays the C code writes into)."""

    def __init__(self, P: int, K: int):
        self.P, self.K = P, K
        self.w = np.zeros((P, K))
        self.mu = np.zeros((P, K, 3))
        self.var = np.zeros((P, K, 3))
        self.rga_m = np.zeros((P, 3))
        self.rga_v = np.zeros((P, 3))
        self.conf = np.zeros(P)
        self.label = np.zeros(P, np.uint8)
        self.prev = np.zeros((P, 3), np.uint8)
        self.kde = np.zeros((P, 3, 256), np.uint8)
        self.qa = np.zeros(P, np.uint8)
        self.qb = np.zeros(P, np.uint8)
        self.illum = np.zeros(2, np.int64)
        self.top = np.zeros(P, np.uint8)
        self.wc = np.zeros((P, 3, K))

    def _c(self) -> _State:
        s = _State()
        for n, _ in _State._fields_:
            a = getattr(self, n)
            assert a.flags.c_contiguous
            setattr(s, n, a.ctypes.data)
        return s

    def copy(self) -> "OracleState":
        o = OracleState(self.P, self.K)
        for n, _ in _State._fields_:
            getattr(o, n)[...] = getattr(self, n)
        return o


class Oracle:
    """One FP64 model of a W x H stream."""

    def __init__(self, params: dict):
        self.p = dict(params)
        self.P = int(params["width"]) * int(params["height"])
        self.K = int(params["K"])
        self.state = OracleState(self.P, self.K)
        self._cp = _params(self.p)
        self.lib = _load()

    def train(self, frames: np.ndarray, want_near: bool = False):
        """Training over frames [N, P, 3].  With want_near, returns the OR
        of the near-threshold bits of every warm-up decision per pixel."""
        f = np.ascontiguousarray(frames, dtype=np.uint8).reshape(-1, self.P, 3)
        s = self.state._c()
        near = np.zeros(self.P, np.uint8) if want_near else None
        if self.lib.orc_train_near(C.byref(self._cp), f.ctypes.data, f.shape[0], C.byref(s),
                                   near.ctypes.data if want_near else None) != 0:
            raise ValueError("orc_train rejected its arguments")
        return near

    def apply(self, frame: np.ndarray, want_stage: bool = True, want_near: bool = True):
        f = np.ascontiguousarray(frame, dtype=np.uint8).reshape(self.P, 3)
        mask = np.empty(self.P, np.uint8)
        stage = np.empty(self.P, np.uint8) if want_stage else None
        near = np.empty(self.P, np.uint8) if want_near else None
        st = _Stats()
        s = self.state._c()
        r = self.lib.orc_apply(C.byref(self._cp), C.byref(s), f.ctypes.data, mask.ctypes.data,
                               stage.ctypes.data if stage is not None else None,
                               near.ctypes.data if near is not None else None, C.byref(st))
        if r != 0:
            raise ValueError("orc_apply rejected its arguments")
        stats = dict(n_stage=list(st.n_stage), n_gmm=int(st.n_gmm), illum_flag=int(st.illum_flag))
        return mask, stage, near, stats

    def group_features(self, frames: np.ndarray):
        """Grouping features over training frames [N, P, 3]: (code_v,
        code_w), the spreads of the dominant mode's mean variance and
        weight over the warm-up, as uint16 codes."""
        f = np.ascontiguousarray(frames, dtype=np.uint8).reshape(-1, self.P, 3)
        cv = np.empty(self.P, np.uint16)
        cw = np.empty(self.P, np.uint16)
        if self.lib.orc_group_features(C.byref(self._cp), f.ctypes.data, f.shape[0], cv.ctypes.data,
                                       cw.ctypes.data) != 0:
            raise ValueError("orc_group_features rejected its arguments")
        return cv, cw

    def group_params(self, labels: np.ndarray) -> dict:
        """Per cluster, the mean over its core pixels (labels & 0x80) of the
        trained state's dominant mode: w1, mu1 [3][3], v1."""
        lab = np.ascontiguousarray(labels, dtype=np.uint8).ravel()
        g = _GroupOut()
        s = self.state._c()
        if self.lib.orc_group_params(C.byref(self._cp), C.byref(s), lab.ctypes.data, C.byref(g)) != 0:
            raise ValueError("orc_group_params rejected its arguments")
        d = _group_dict(g)
        return dict(w1=d["w1"], mu1=d["mu1"], v1=d["v1"])

    def plain_gmm(self, w: np.ndarray, mu: np.ndarray, var: np.ndarray, frame: np.ndarray):
        for a in (w, mu, var):
            assert a.dtype == np.float64 and a.flags.c_contiguous
        f = np.ascontiguousarray(frame, dtype=np.uint8).reshape(self.P, 3)
        mask = np.empty(self.P, np.uint8)
        r = self.lib.orc_plain_gmm(C.byref(self._cp), w.ctypes.data, mu.ctypes.data,
                                   var.ctypes.data, f.ctypes.data, mask.ctypes.data)
        if r != 0:
            raise ValueError("orc_plain_gmm rejected its arguments")
        return mask
