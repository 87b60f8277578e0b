"""Thin ctypes binding of libnb (include/nb.h) over PyTorch device tensors.

Argument marshalling only: every step of the hot path runs in libnb's CUDA kernels.
PyTorch provides device memory and the current stream.  There is no CPU fallback:
if libnb.so cannot be loaded the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

from . import build as _build
from .inputs import ENC_WIDTH, POINT2, POINT4T

NB_F32, NB_BF16, NB_FP8, NB_F16X3 = 0, 1, 2, 3
PREC = {"f32": NB_F32, "bf16": NB_BF16, "fp8": NB_FP8, "f16x3": NB_F16X3}
ACT = {"relu": 0, "sine": 1}  # NB_ACT_RELU, NB_ACT_SINE
STATUS = {0: "NB_OK", 1: "NB_EINVAL", 2: "NB_ENOMEM", 3: "NB_ECUDA", 4: "NB_ETIMEOUT", 5: "NB_ENUMERIC",
          6: "NB_EUNSUPPORTED"}

# every symbol include/nb.h declares
EXPORTS = ["nb_model_create", "nb_model_create_act", "nb_model_destroy", "nb_model_param_count", "nb_model_set_params",
           "nb_model_get_params", "nb_model_get_grad", "nb_model_set_tau", "nb_model_get_tau",
           "nb_model_set_adam", "nb_model_state_size", "nb_model_get_state", "nb_model_set_state",
           "nb_label", "nb_train_step", "nb_query", "nb_calibrate", "nb_last_error", "nb_train_step_noalloc",
           "nb_plan_create", "nb_plan_destroy", "nb_group_create", "nb_group_destroy", "nb_group_param_count",
           "nb_group_set_params", "nb_group_get_params", "nb_group_get_grad", "nb_group_set_tau", "nb_group_get_tau",
           "nb_group_set_schedule", "nb_group_sync_schedule", "nb_group_reserve", "nb_train_step_grouped",
           "nb_query_grouped", "nb_calibrate_grouped", "nb_cascade_bin", "nb_cascade_exact", "nb_sample", "nb_group_autotune", "nb_query_early_out", "nb_bits_not",
           "nb_query_three_way", "nb_cascade_index_create", "nb_cascade_index_destroy", "nb_cascade_bin_indexed",
           "nb_cascade_index_max_nodes", "nb_cascade_index_build_host", "nb_stepwise_init", "nb_stepwise_window",
           "nb_query_host", "nb_model_check", "nb_selftest_bounded_wait", "nb_encode_paper"]


class NBError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Shape(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("n_spheres", ctypes.c_int32), ("qexp", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("centres", ctypes.c_void_p), ("radii", ctypes.c_void_p),
                ("vel", ctypes.c_void_p)]


LABEL_STATS = np.dtype([("n_positive", "<u8"), ("n_invalid", "<u8")])
QUERY_STATS = np.dtype([("n_inside", "<u8"), ("n_flagged", "<u8"), ("n_resolved_f32", "<u8"),
                        ("n_resolved_ff", "<u8"), ("n_unresolved", "<u8"), ("n_nonfinite", "<u8")])
STEP_STATS = np.dtype([("loss", "<f4"), ("reserved", "<f4"), ("fn", "<u8"), ("fp", "<u8"),
                       ("n_nonfinite", "<u8")])

_lock = threading.Lock()
_lib = None


def lib():
    """Load libnb.so (building it in-tree first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if _build._stale():
                path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError("libnb.so is not built; run paper_2310_06822_gb300/build.py")
            L = ctypes.CDLL(path)
            P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
            st = ctypes.c_int
            sig = {
                "nb_model_create": ([P, i32, i32, i32, P], st),
                "nb_model_create_act": ([P, i32, i32, i32, i32, P], st),
                "nb_model_destroy": ([P], st),
                "nb_model_param_count": ([P], i64),
                "nb_model_set_params": ([P, P, i64], st),
                "nb_model_get_params": ([P, P, i64], st),
                "nb_model_get_grad": ([P, P, i64], st),
                "nb_model_set_tau": ([P, ctypes.c_double], st),
                "nb_model_get_tau": ([P, P], st),
                "nb_model_set_adam": ([P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float], st),
                "nb_model_state_size": ([P, P], st),
                "nb_model_get_state": ([P, P, ctypes.c_size_t], st),
                "nb_model_set_state": ([P, P, ctypes.c_size_t], st),
                "nb_label": ([P, i32, P, i64, P, P, P], st),
                "nb_train_step": ([P, P, P, i64, ctypes.c_float, ctypes.c_float, P, P], st),
                "nb_query": ([P, P, i64, ctypes.c_float, P, P, P, P], st),
                "nb_calibrate": ([P, P, P, i64, ctypes.c_double, P, P], st),
                "nb_last_error": ([], ctypes.c_char_p),
                "nb_train_step_noalloc": ([P, P, P, i64, ctypes.c_float, ctypes.c_float, P, P], st),
                "nb_plan_create": ([P, i32, i32, P], st),
                "nb_plan_destroy": ([P], st),
                "nb_group_create": ([P, i32, i32, i32, i32, P], st),
                "nb_group_destroy": ([P], st),
                "nb_group_param_count": ([P], i64),
                "nb_group_set_params": ([P, P, i64], st),
                "nb_group_get_params": ([P, P, i64], st),
                "nb_group_get_grad": ([P, P, i64], st),
                "nb_group_set_tau": ([P, P, i32], st),
                "nb_group_get_tau": ([P, P, i32], st),
                "nb_group_set_schedule": ([P, P, i32], st),
                "nb_group_sync_schedule": ([P], st),
                "nb_group_reserve": ([P, P], st),
                "nb_train_step_grouped": ([P, P, P, P, ctypes.c_float, ctypes.c_float, P, P], st),
                "nb_query_grouped": ([P, P, P, ctypes.c_float, P, P, P, P], st),
                "nb_calibrate_grouped": ([P, P, P, P, ctypes.c_double, P, P], st),
                "nb_cascade_bin": ([P, P, i64, i32, P, P, P, P, P, P], st),
                "nb_cascade_exact": ([P, P, P, P, i64, P, P, P, P, P], st),
                "nb_sample": ([i32, i32, ctypes.c_uint64, i64, i64, P, P], st),
                "nb_group_autotune": ([P, P, i32, i32, P, P, P, i32, i32, P, P, P], st),
                "nb_query_early_out": ([P, P, P, i64, ctypes.c_float, ctypes.c_float, P, P, P], st),
                "nb_bits_not": ([P, i64, P, P], st),
                "nb_query_three_way": ([P, P, P, i64, ctypes.c_float, ctypes.c_float, P, P, P], st),
                "nb_cascade_index_create": ([P, P], st),
                "nb_cascade_index_destroy": ([P], st),
                "nb_cascade_bin_indexed": ([P, P, P, i64, i32, P, P, P, P, P, P], st),
                "nb_cascade_index_max_nodes": ([i32], i32),
                "nb_cascade_index_build_host": ([P, i32, P, P, P], st),
                "nb_stepwise_init": ([P, i32, i32, ctypes.c_float, i32], st),
                "nb_stepwise_window": ([P, ctypes.c_uint64], i32),
                "nb_query_host": ([P, P, i64, ctypes.c_float, P, P, i64, P], st),
                "nb_model_check": ([P, P], st),
                "nb_selftest_bounded_wait": ([i32, P], st),
                "nb_encode_paper": ([i32, P, i64, P, P], st),
            }
            for name, (args, res) in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def _check(rc):
    if rc != 0:
        msg = lib().nb_last_error()
        raise NBError(rc, msg.decode() if msg else "")


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _dev(x, dtype, device="cuda"):
    if isinstance(x, torch.Tensor):
        t = x.to(device=device, dtype=dtype)
    else:
        t = torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device=device)
    return t.contiguous()


def n_words(n: int) -> int:
    return (n + 31) // 32


def _read(t: torch.Tensor, dt: np.dtype) -> dict:
    a = np.frombuffer(t.cpu().numpy().tobytes(), dtype=dt)[0]
    return {k: (float(a[k]) if a[k].dtype.kind == "f" else int(a[k])) for k in dt.names if k != "reserved"}


class Shape:
    """A union of spheres resident on the device (nb_shape)."""

    def __init__(self, scene, device="cuda"):
        self.scene = scene
        self.centres = _dev(scene.centres, torch.float32, device)
        self.radii = _dev(scene.radii, torch.float32, device)
        self.vel = None if scene.vel is None else _dev(scene.vel, torch.float32, device)
        self._s = _Shape(scene.dim, scene.n_spheres, scene.qexp, 0, self.centres.data_ptr(),
                         self.radii.data_ptr(), self.vel.data_ptr() if self.vel is not None else None)


def sample(kind: int, n: int, seed: int, first: int = 0, qexp: int = 20, out: torch.Tensor | None = None,
           device="cuda", stream=None) -> torch.Tensor:
    """Queries first .. first+n-1 of the counter-based stream (seed, kind) (nb_sample)."""
    if out is None:
        out = torch.empty((n, ENC_WIDTH[kind]), dtype=torch.float32, device=device)
    _check(lib().nb_sample(int(kind), int(qexp), int(seed), int(first), int(n), _ptr(out), _stream(stream)))
    return out


def label(shape: Shape, kind: int, q: torch.Tensor, out: torch.Tensor | None = None, stats: bool = False,
          stream=None):
    """Exact labels of n queries (packed bits, int32 words) via nb_label."""
    n = q.shape[0]
    if out is None:
        out = torch.empty(n_words(n), dtype=torch.int32, device=q.device)
    st = torch.empty(LABEL_STATS.itemsize, dtype=torch.uint8, device=q.device) if stats else None
    _check(lib().nb_label(ctypes.byref(shape._s), int(kind), _ptr(q), n, _ptr(out), _ptr(st), _stream(stream)))
    if stats:
        return out, _read(st, LABEL_STATS)
    return out


class Model:
    """A bounding network h (nb_model)."""

    def __init__(self, widths, infer_prec="f32", train_prec="f32", activation="relu"):
        self.widths = [int(w) for w in widths]
        self.infer_prec = PREC[infer_prec] if isinstance(infer_prec, str) else int(infer_prec)
        self.train_prec = PREC[train_prec] if isinstance(train_prec, str) else int(train_prec)
        self.activation = ACT[activation] if isinstance(activation, str) else int(activation)
        w = (ctypes.c_int32 * len(self.widths))(*self.widths)
        h = ctypes.c_void_p()
        _check(lib().nb_model_create_act(w, len(self.widths) - 1, self.infer_prec, self.train_prec, self.activation,
                                         ctypes.byref(h)))
        self._h = h
        self.P = int(lib().nb_model_param_count(h))

    def close(self):
        if getattr(self, "_h", None):
            lib().nb_model_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- state
    def set_params(self, p):
        p = np.ascontiguousarray(np.asarray(p, dtype=np.float32))
        _check(lib().nb_model_set_params(self._h, p.ctypes.data_as(ctypes.c_void_p), p.size))

    def get_params(self) -> np.ndarray:
        p = np.zeros(self.P, dtype=np.float32)
        _check(lib().nb_model_get_params(self._h, p.ctypes.data_as(ctypes.c_void_p), self.P))
        return p

    def get_grad(self) -> np.ndarray:
        g = np.zeros(self.P, dtype=np.float32)
        _check(lib().nb_model_get_grad(self._h, g.ctypes.data_as(ctypes.c_void_p), self.P))
        return g

    @property
    def tau(self) -> float:
        t = ctypes.c_double()
        _check(lib().nb_model_get_tau(self._h, ctypes.byref(t)))
        return t.value

    @tau.setter
    def tau(self, v: float):
        _check(lib().nb_model_set_tau(self._h, float(v)))

    def set_adam(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        _check(lib().nb_model_set_adam(self._h, lr, b1, b2, eps))

    def get_state(self) -> bytes:
        n = ctypes.c_size_t()
        _check(lib().nb_model_state_size(self._h, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        _check(lib().nb_model_get_state(self._h, buf, n.value))
        return buf.raw

    def set_state(self, b: bytes):
        buf = ctypes.create_string_buffer(b, len(b))
        _check(lib().nb_model_set_state(self._h, buf, len(b)))

    # -- hot path
    def train_step(self, q, label_bits, alpha: float, beta: float = 1.0, stats=None, stream=None):
        """One fused training iteration; stats (a uint8 device tensor of 32 bytes) optional."""
        _check(lib().nb_train_step(self._h, _ptr(q), _ptr(label_bits), q.shape[0], float(alpha), float(beta),
                                   _ptr(stats), _stream(stream)))

    def query(self, q, margin: float = 0.0, out=None, logits: bool = False, stats: bool = False, stream=None):
        n = q.shape[0]
        if out is None:
            out = torch.empty(n_words(n), dtype=torch.int32, device=q.device)
        lg = torch.empty(n, dtype=torch.float32, device=q.device) if logits else None
        st = torch.empty(QUERY_STATS.itemsize, dtype=torch.uint8, device=q.device) if stats else None
        _check(lib().nb_query(self._h, _ptr(q), n, float(margin), _ptr(out), _ptr(lg), _ptr(st), _stream(stream)))
        res = [out]
        if logits:
            res.append(lg)
        if stats:
            res.append(_read(st, QUERY_STATS))
        return res[0] if len(res) == 1 else tuple(res)

    def calibrate(self, q, label_bits, eps: float = 1e-5, stream=None) -> float:
        t = ctypes.c_double()
        _check(lib().nb_calibrate(self._h, _ptr(q), _ptr(label_bits), q.shape[0], float(eps), ctypes.byref(t),
                                  _stream(stream)))
        return t.value

    def check(self, stream=None):
        """Raise NBError if the model's asynchronous work failed (nb_model_check)."""
        _check(lib().nb_model_check(self._h, _stream(stream)))

    def query_host(self, q, margin: float = 0.0, out=None, stats: bool = False, chunk_rows: int = 0, stream=None):
        """Decisions for queries in host memory (nb_query_host): q a contiguous float32 CPU
        tensor (pinned for copy/compute overlap), the bits into a CPU int32 tensor."""
        if q.is_cuda or q.dtype != torch.float32 or not q.is_contiguous():
            raise ValueError("q must be a contiguous float32 host tensor")
        n = q.shape[0]
        if out is None:
            out = torch.empty(n_words(n), dtype=torch.int32, pin_memory=q.is_pinned())
        st = np.zeros(1, dtype=QUERY_STATS)
        _check(lib().nb_query_host(self._h, _ptr(q), n, float(margin), _ptr(out),
                                   st.ctypes.data_as(ctypes.c_void_p) if stats else None, int(chunk_rows),
                                   _stream(stream)))
        if stats:
            return out, {k: int(st[0][k]) for k in QUERY_STATS.names}
        return out


class Plan:
    """Work items over concatenated per-object rows (nb_plan)."""

    def __init__(self, offsets, chunk_rows: int = 0):
        off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        self.offsets = off
        self.n_objects = len(off) - 1
        self.n_rows = int(off[-1])
        h = ctypes.c_void_p()
        _check(lib().nb_plan_create(off.ctypes.data_as(ctypes.c_void_p), self.n_objects, int(chunk_rows),
                                    ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().nb_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Group:
    """n_objects bounding networks of one architecture (nb_group)."""

    def __init__(self, widths, n_objects: int, infer_prec="f32", train_prec="f32"):
        self.widths = [int(w) for w in widths]
        self.n_objects = int(n_objects)
        ip = PREC[infer_prec] if isinstance(infer_prec, str) else int(infer_prec)
        tp = PREC[train_prec] if isinstance(train_prec, str) else int(train_prec)
        w = (ctypes.c_int32 * len(self.widths))(*self.widths)
        h = ctypes.c_void_p()
        _check(lib().nb_group_create(w, len(self.widths) - 1, self.n_objects, ip, tp, ctypes.byref(h)))
        self._h = h
        self.P = int(lib().nb_group_param_count(h))

    def close(self):
        if getattr(self, "_h", None):
            lib().nb_group_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, p):
        p = np.ascontiguousarray(np.asarray(p, dtype=np.float32).ravel())
        _check(lib().nb_group_set_params(self._h, p.ctypes.data_as(ctypes.c_void_p), p.size))

    def get_params(self) -> np.ndarray:
        p = np.zeros(self.P * self.n_objects, dtype=np.float32)
        _check(lib().nb_group_get_params(self._h, p.ctypes.data_as(ctypes.c_void_p), p.size))
        return p.reshape(self.n_objects, self.P)

    def get_grad(self) -> np.ndarray:
        g = np.zeros(self.P * self.n_objects, dtype=np.float32)
        _check(lib().nb_group_get_grad(self._h, g.ctypes.data_as(ctypes.c_void_p), g.size))
        return g.reshape(self.n_objects, self.P)

    @property
    def tau(self) -> np.ndarray:
        t = np.zeros(self.n_objects, dtype=np.float64)
        _check(lib().nb_group_get_tau(self._h, t.ctypes.data_as(ctypes.c_void_p), self.n_objects))
        return t

    @tau.setter
    def tau(self, v):
        t = np.ascontiguousarray(np.broadcast_to(np.asarray(v, dtype=np.float64), (self.n_objects,)))
        _check(lib().nb_group_set_tau(self._h, t.ctypes.data_as(ctypes.c_void_p), self.n_objects))

    def set_schedule(self, alpha):
        a = np.ascontiguousarray(np.asarray(alpha, dtype=np.float32))
        _check(lib().nb_group_set_schedule(self._h, a.ctypes.data_as(ctypes.c_void_p), a.size))

    def sync_schedule(self):
        _check(lib().nb_group_sync_schedule(self._h))

    def reserve(self, plan: Plan):
        _check(lib().nb_group_reserve(self._h, plan._h))

    def train_step(self, plan: Plan, q, label_bits, alpha: float, beta: float = 1.0, stats=None, stream=None):
        _check(lib().nb_train_step_grouped(self._h, plan._h, _ptr(q), _ptr(label_bits), float(alpha), float(beta),
                                           _ptr(stats), _stream(stream)))

    def query(self, plan: Plan, q, margin: float = 0.0, out=None, logits: bool = False, stats: bool = False,
              stream=None):
        n = plan.n_rows
        if out is None:
            out = torch.empty(n_words(n), dtype=torch.int32, device=q.device)
        lg = torch.empty(n, dtype=torch.float32, device=q.device) if logits else None
        st = torch.empty(QUERY_STATS.itemsize, dtype=torch.uint8, device=q.device) if stats else None
        _check(lib().nb_query_grouped(self._h, plan._h, _ptr(q), float(margin), _ptr(out), _ptr(lg), _ptr(st),
                                      _stream(stream)))
        res = [out]
        if logits:
            res.append(lg)
        if stats:
            res.append(_read(st, QUERY_STATS))
        return res[0] if len(res) == 1 else tuple(res)

    def autotune(self, offsets, q, label_bits=None, op: str = "query", candidates=(1024, 2048, 4096, 8192, 16384),
                 reps: int = 3, stream=None):
        """Fastest chunk_rows of the candidates for the grouped query or training step on
        these rows (nb_group_autotune); returns (best, {candidate: ms})."""
        off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        cand = np.ascontiguousarray(np.asarray(candidates, dtype=np.int32))
        ms = np.zeros(cand.size, dtype=np.float32)
        best = ctypes.c_int32(0)
        _check(lib().nb_group_autotune(self._h, off.ctypes.data_as(ctypes.c_void_p), self.n_objects,
                                       {"query": 0, "train": 1}[op], _ptr(q), _ptr(label_bits),
                                       cand.ctypes.data_as(ctypes.c_void_p), cand.size, int(reps), ctypes.byref(best),
                                       ms.ctypes.data_as(ctypes.c_void_p), _stream(stream)))
        return int(best.value), {int(c): float(m) for c, m in zip(cand, ms)}

    def calibrate(self, plan: Plan, q, label_bits, eps: float = 1e-5, stream=None) -> np.ndarray:
        t = np.zeros(self.n_objects, dtype=np.float64)
        _check(lib().nb_calibrate_grouped(self._h, plan._h, _ptr(q), _ptr(label_bits), float(eps),
                                          t.ctypes.data_as(ctypes.c_void_p), _stream(stream)))
        return t


class _SceneC(ctypes.Structure):
    _fields_ = [("n_objects", ctypes.c_int32), ("qexp", ctypes.c_int32), ("ball_radius", ctypes.c_float),
                ("reserved", ctypes.c_int32), ("sphere_offsets", ctypes.c_void_p), ("centres", ctypes.c_void_p),
                ("radii", ctypes.c_void_p), ("obj_centre", ctypes.c_void_p), ("aabb", ctypes.c_void_p)]


CASCADE_STATS = np.dtype([("aabb_pairs", "<u8"), ("ball_pairs", "<u8"), ("exact_pairs", "<u8"),
                          ("sphere_tests", "<u8"), ("hit_pairs", "<u8")])


class WorldScene:
    """Objects of a multi-object scene resident on the device (nb_scene)."""

    def __init__(self, ms, device="cuda"):
        self.ms = ms
        self.K = ms.n_objects
        self.sphere_offsets = torch.as_tensor(np.ascontiguousarray(ms.sphere_offsets, dtype=np.int64), device=device)
        self.centres = _dev(ms.centres, torch.float32, device)
        self.radii = _dev(ms.radii, torch.float32, device)
        self.obj_centre = _dev(ms.obj_centre, torch.float32, device)
        self.aabb = _dev(ms.aabb, torch.float32, device)
        self._s = _SceneC(self.K, ms.qexp, float(ms.ball_radius), 0, self.sphere_offsets.data_ptr(),
                          self.centres.data_ptr(), self.radii.data_ptr(), self.obj_centre.data_ptr(),
                          self.aabb.data_ptr())


BVH4_NODE = np.dtype([("lo", "<f4", (3, 4)), ("hi", "<f4", (3, 4)), ("child", "<i4", (4,))])
BVH_EMPTY = -2 ** 31


def bvh4_build_host(aabb: np.ndarray):
    """The object tree of the cascade index built on the host (nb_cascade_index_build_host):
    returns (nodes as a BVH4_NODE array, depth).  No device is involved."""
    a = np.ascontiguousarray(aabb, dtype=np.float32).reshape(-1, 6)
    K = a.shape[0]
    L = lib()
    nodes = np.zeros(max(1, L.nb_cascade_index_max_nodes(K)), dtype=BVH4_NODE)
    nn, dep = ctypes.c_int32(0), ctypes.c_int32(0)
    _check(L.nb_cascade_index_build_host(a.ctypes.data_as(ctypes.c_void_p), K,
                                         nodes.ctypes.data_as(ctypes.c_void_p), ctypes.byref(nn), ctypes.byref(dep)))
    return nodes[:nn.value].copy(), dep.value


class CascadeIndex:
    """Spatial index (4-wide tree of object boxes) of a WorldScene, for stage 1."""

    def __init__(self, ws: WorldScene):
        self.ws = ws
        h = ctypes.c_void_p()
        _check(lib().nb_cascade_index_create(ctypes.byref(ws._s), ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().nb_cascade_index_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cascade_bin(ws: WorldScene, rays: torch.Tensor, canonical: bool, stream=None, index: CascadeIndex | None = None):
    """Stage 1: (ray, object) pairs passing the box (and the ball when canonical), binned by
    object into rows padded to multiples of 32, through the spatial index when one is
    given.  Returns (host offsets, device offsets, pair_ray, pair_q or None, stats)."""
    n = rays.shape[0]
    dev = rays.device
    counts = torch.zeros(ws.K, dtype=torch.int64, device=dev)
    st = torch.zeros(CASCADE_STATS.itemsize, dtype=torch.uint8, device=dev)
    L = lib()

    def call(off_d, pair_ray, pair_q, stats):
        if index is None:
            return L.nb_cascade_bin(ctypes.byref(ws._s), _ptr(rays), n, int(canonical), _ptr(counts), _ptr(off_d),
                                    _ptr(pair_ray), _ptr(pair_q), _ptr(stats), _stream(stream))
        return L.nb_cascade_bin_indexed(index._h, ctypes.byref(ws._s), _ptr(rays), n, int(canonical), _ptr(counts),
                                        _ptr(off_d), _ptr(pair_ray), _ptr(pair_q), _ptr(stats), _stream(stream))

    _check(call(None, None, None, st))
    c = counts.cpu().numpy()
    padded = (c + 31) // 32 * 32
    off = np.concatenate([[0], np.cumsum(padded)]).astype(np.int64)
    rows = int(off[-1])
    pair_ray = torch.full((max(rows, 1),), -1, dtype=torch.int32, device=dev)
    pair_q = torch.zeros((max(rows, 1), 6), dtype=torch.float32, device=dev) if canonical else None
    off_d = torch.as_tensor(off, device=dev)
    _check(call(off_d, pair_ray, pair_q, None))
    return off, off_d, pair_ray, pair_q, _read(st, CASCADE_STATS)


def cascade_exact(ws: WorldScene, rays, pair_ray, off_d, rows: int, pass_bits=None, ray_hits=None,
                  pair_hits=None, stats=None, stream=None):
    """Stage 3: exact sphere tests of the rows (those with a pass bit, if given)."""
    _check(lib().nb_cascade_exact(ctypes.byref(ws._s), _ptr(rays), _ptr(pair_ray), _ptr(off_d), int(rows),
                                  _ptr(pass_bits), _ptr(ray_hits), _ptr(pair_hits), _ptr(stats), _stream(stream)))


def bits_not(bits: torch.Tensor, n: int, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """The complement of n label or decision bits (nb_bits_not)."""
    if out is None:
        out = torch.empty_like(bits)
    _check(lib().nb_bits_not(_ptr(bits), int(n), _ptr(out), _stream(stream)))
    return out


def query_early_out(early: Model, late: Model, q: torch.Tensor, margin_early: float = 0.0, margin_late: float = 0.0,
                    out: torch.Tensor | None = None, stream=None):
    """Decisions with the neural early-out (nb_query_early_out); returns (bits, stats)."""
    n = q.shape[0]
    if out is None:
        out = torch.empty(n_words(n), dtype=torch.int32, device=q.device)
    st = (ctypes.c_uint64 * 2)()
    _check(lib().nb_query_early_out(early._h, late._h, _ptr(q), n, float(margin_early), float(margin_late),
                                    _ptr(out), ctypes.byref(st), _stream(stream)))
    return out, {"n_early_inside": int(st[0]), "n_late": int(st[1])}


THREE_WAY_OUT, THREE_WAY_IN, THREE_WAY_NEITHER = 0, 1, 2


def query_three_way(outer: Model, inner: Model, q: torch.Tensor, margin_outer: float = 0.0,
                    margin_inner: float = 0.0, out: torch.Tensor | None = None, stats: torch.Tensor | None = None,
                    stream=None) -> torch.Tensor:
    """Broad-phase class of each query from a bound (outer) and a bound of the complement
    (inner) (nb_query_three_way): uint8 codes 0 certainly outside, 1 certainly inside,
    2 neither.  stats, if given, is a device uint64 tensor of 4 (out, in, neither,
    conflicts) that is added to."""
    n = q.shape[0]
    if out is None:
        out = torch.empty(n, dtype=torch.uint8, device=q.device)
    if stats is not None and (stats.dtype != torch.int64 or stats.numel() < 4 or not stats.is_cuda):
        raise ValueError("stats must be a device int64 tensor of 4")
    _check(lib().nb_query_three_way(outer._h, inner._h, _ptr(q), n, float(margin_outer), float(margin_inner),
                                    _ptr(out), _ptr(stats), _stream(stream)))
    return out


class _StepwiseC(ctypes.Structure):
    _fields_ = [("period", ctypes.c_int32), ("dim_rate", ctypes.c_int32), ("fn_step", ctypes.c_float),
                ("stop_windows", ctypes.c_int32), ("adjustments", ctypes.c_int32), ("clean_windows", ctypes.c_int32),
                ("alpha", ctypes.c_float), ("beta", ctypes.c_float)]


class Stepwise:
    """Stepwise asymmetry schedule of the loss weights (nb_stepwise_*): alpha and beta
    change at the end of a window of `period` steps that saw false negatives."""

    RATES = {2: 20, 3: 100, 4: 200}

    def __init__(self, dim: int = 3, period: int = 10000, fn_step: float = 0.2, stop_windows: int = 0,
                 dim_rate: int | None = None):
        self._s = _StepwiseC()
        rate = dim_rate if dim_rate is not None else self.RATES[dim]
        _check(lib().nb_stepwise_init(ctypes.byref(self._s), int(period), int(rate), float(fn_step),
                                      int(stop_windows)))

    @property
    def alpha(self) -> float:
        return self._s.alpha

    @property
    def beta(self) -> float:
        return self._s.beta

    @property
    def period(self) -> int:
        return self._s.period

    @property
    def adjustments(self) -> int:
        return self._s.adjustments

    def window(self, fn: int) -> bool:
        """End of a window with fn false negatives; True when training may stop."""
        r = lib().nb_stepwise_window(ctypes.byref(self._s), int(fn))
        if r < 0:
            raise NBError(1, "nb_stepwise_window: uninitialised schedule")
        return r == 1


PAPER_ENC_WIDTH = (2, 3, 4, 6, 6, 6)


def encode_paper(kind: int, q: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """The paper's query parameterisation of q (nb_encode_paper): box corners, plane point
    and normal; rays and points unchanged."""
    n = q.shape[0]
    if out is None:
        out = torch.empty((n, PAPER_ENC_WIDTH[kind]), dtype=torch.float32, device=q.device)
    _check(lib().nb_encode_paper(int(kind), _ptr(q), n, _ptr(out), _stream(stream)))
    return out


def selftest_bounded_wait(polls: int = 1024, stream=None) -> int:
    """Status of one bounded device wait that nothing completes (NB_ETIMEOUT expected)."""
    return int(lib().nb_selftest_bounded_wait(int(polls), _stream(stream)))


def step_stats_tensor(device="cuda") -> torch.Tensor:
    return torch.zeros(STEP_STATS.itemsize, dtype=torch.uint8, device=device)


def read_step_stats(t: torch.Tensor) -> dict:
    return _read(t, STEP_STATS)


def bits_to_numpy(words: torch.Tensor, n: int) -> np.ndarray:
    from .inputs import unpack_bits
    return unpack_bits(words.cpu().numpy().view(np.uint32), n)


def numpy_bits_to_device(words: np.ndarray, device="cuda") -> torch.Tensor:
    return torch.as_tensor(np.ascontiguousarray(words).view(np.int32), device=device)


def enc_width(kind: int) -> int:
    return ENC_WIDTH[kind]


__all__ = ["Model", "Group", "Plan", "Shape", "label", "lib", "NBError", "EXPORTS", "POINT2", "POINT4T"]
