"""ctypes front end of the FP64 / exact-integer CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  The product library never imports this.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
SO = os.path.join(OUT_DIR, "liboracle.so")

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (no fast-math, no FMA contraction)."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(SO) and os.path.getmtime(SO) >= os.path.getmtime(SRC):
        return SO
    tmp = SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fno-fast-math", "-ffp-contract=off", "-frounding-math",
           "-shared", "-fPIC", "-pthread", SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, SO)
    return SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(SO)
            P = ctypes.c_void_p
            i64 = ctypes.c_int64
            L.orc_label.argtypes = [ctypes.c_int, P, i64, ctypes.c_int, ctypes.c_int, P, P, P,
                                    ctypes.c_int, P, ctypes.c_int]
            L.orc_label.restype = ctypes.c_int
            L.orc_mc_label.argtypes = [ctypes.c_int, P, i64, ctypes.c_int, P, P, ctypes.c_int,
                                       ctypes.c_int, P]
            L.orc_mc_label.restype = ctypes.c_int
            L.orc_param_count.argtypes = [P, ctypes.c_int]
            L.orc_param_count.restype = i64
            L.orc_forward.argtypes = [P, ctypes.c_int, P, P, i64, P, ctypes.c_int]
            L.orc_forward.restype = ctypes.c_int
            L.orc_forward_scale.argtypes = [P, ctypes.c_int, P, P, i64, P]
            L.orc_forward_scale.restype = ctypes.c_int
            L.orc_loss_grad.argtypes =[P, ctypes.c_int, P, P, P, i64, ctypes.c_double,
                                        ctypes.c_double, P, P, ctypes.c_int]
            L.orc_loss_grad.restype = ctypes.c_int
            L.orc_adam.argtypes = [i64, P, P, P, P, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_double, i64]
            L.orc_adam.restype = None
            L.orc_calibrate.argtypes = [P, P, i64, ctypes.c_double, P]
            L.orc_calibrate.restype = i64
            L.orc_count.argtypes = [P, P, i64, ctypes.c_double, P]
            L.orc_count.restype = None
            L.orc_philox4x64.argtypes = [P, P, P]
            L.orc_philox4x64.restype = None
            L.orc_sample.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint64, i64, i64, P, ctypes.c_int]
            L.orc_sample.restype = ctypes.c_int
            L.orc_forward_act.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P, i64, P, ctypes.c_int]
            L.orc_forward_act.restype = ctypes.c_int
            L.orc_forward_scale_act.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P, i64, P]
            L.orc_forward_scale_act.restype = ctypes.c_int
            L.orc_loss_grad_act.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P, P, i64, ctypes.c_double,
                                            ctypes.c_double, P, P, ctypes.c_int]
            L.orc_loss_grad_act.restype = ctypes.c_int
            L.orc_canonical_ray.argtypes = [P, P, i64, ctypes.c_float, P, P]
            L.orc_canonical_ray.restype = ctypes.c_int
            L.orc_canonical_ray_f64.argtypes = [P, P, i64, ctypes.c_double, P, P]
            L.orc_canonical_ray_f64.restype = ctypes.c_int
            _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _threads(nthreads):
    return int(nthreads) if nthreads else (os.cpu_count() or 1)


def label(kind: int, q: np.ndarray, scene, nthreads: int | None = None) -> np.ndarray:
    """Exact labels (uint8 0/1) of ``n`` queries against ``scene`` (inputs.Scene)."""
    q = np.ascontiguousarray(q, dtype=np.float32)
    c = np.ascontiguousarray(scene.centres, dtype=np.float32)
    r = np.ascontiguousarray(scene.radii, dtype=np.float32)
    v = None if scene.vel is None else np.ascontiguousarray(scene.vel, dtype=np.float32)
    n = q.shape[0]
    out = np.zeros(n, dtype=np.uint8)
    rc = lib().orc_label(int(kind), _ptr(q), n, c.shape[1], r.shape[0], _ptr(c), _ptr(r), _ptr(v),
                         int(scene.qexp), _ptr(out), _threads(nthreads))
    if rc != 0:
        raise ValueError("oracle label: input off the grid, non-finite or malformed")
    return out


def mc_label(kind: int, q: np.ndarray, scene, density: int) -> np.ndarray:
    """Alg. 1 labels: any() of the indicator over a lattice sample of each region."""
    q = np.ascontiguousarray(q, dtype=np.float32)
    c = np.ascontiguousarray(scene.centres, dtype=np.float32)
    r = np.ascontiguousarray(scene.radii, dtype=np.float32)
    out = np.zeros(q.shape[0], dtype=np.uint8)
    rc = lib().orc_mc_label(int(kind), _ptr(q), q.shape[0], r.shape[0], _ptr(c), _ptr(r),
                            int(scene.qexp), int(density), _ptr(out))
    if rc != 0:
        raise ValueError("oracle mc_label failed")
    return out


def param_count(widths) -> int:
    w = np.ascontiguousarray(widths, dtype=np.int32)
    return int(lib().orc_param_count(_ptr(w), len(widths) - 1))


ACTS = {"relu": 0, "sine": 1}


def forward(widths, params: np.ndarray, X: np.ndarray, nthreads: int | None = None, act: str = "relu") -> np.ndarray:
    """FP64 logits z of the MLP on the FP32 parameters (hidden activation ReLU or sine)."""
    w = np.ascontiguousarray(widths, dtype=np.int32)
    p = np.ascontiguousarray(params, dtype=np.float32)
    X = np.ascontiguousarray(X, dtype=np.float32)
    z = np.zeros(X.shape[0], dtype=np.float64)
    rc = lib().orc_forward_act(_ptr(w), len(widths) - 1, ACTS[act], _ptr(p), _ptr(X), X.shape[0], _ptr(z),
                               _threads(nthreads))
    if rc != 0:
        raise ValueError("oracle forward: bad widths")
    return z


def forward_scale(widths, params: np.ndarray, X: np.ndarray, act: str = "relu") -> np.ndarray:
    """sum_k |W_L[k]| a_{L-1}[k] + |b_L| per query (FP64): the scale the last layer's
    rounding error is relative to."""
    w = np.ascontiguousarray(widths, dtype=np.int32)
    p = np.ascontiguousarray(params, dtype=np.float32)
    X = np.ascontiguousarray(X, dtype=np.float32)
    s = np.zeros(X.shape[0], dtype=np.float64)
    if lib().orc_forward_scale_act(_ptr(w), len(widths) - 1, ACTS[act], _ptr(p), _ptr(X), X.shape[0], _ptr(s)) != 0:
        raise ValueError("oracle forward_scale: bad widths")
    return s


def loss_grad(widths, params, X, y, alpha: float, beta: float, nthreads: int | None = None, act: str = "relu"):
    """Mean asymmetric BCE (Eq. loss) and its FP64 gradient w.r.t. the flat parameters."""
    w = np.ascontiguousarray(widths, dtype=np.int32)
    p = np.ascontiguousarray(params, dtype=np.float32)
    X = np.ascontiguousarray(X, dtype=np.float32)
    y = np.ascontiguousarray(np.asarray(y).astype(np.uint8))
    g = np.zeros(p.shape[0], dtype=np.float64)
    loss = np.zeros(1, dtype=np.float64)
    rc = lib().orc_loss_grad_act(_ptr(w), len(widths) - 1, ACTS[act], _ptr(p), _ptr(X), _ptr(y), X.shape[0],
                                 float(alpha), float(beta), _ptr(loss), _ptr(g), _threads(nthreads))
    if rc != 0:
        raise ValueError("oracle loss_grad failed")
    return float(loss[0]), g


def adam(theta, m, v, g, t: int, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (in place on float64 arrays theta, m, v)."""
    for a in (theta, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = np.ascontiguousarray(g, dtype=np.float64)
    lib().orc_adam(theta.shape[0], _ptr(theta), _ptr(m), _ptr(v), _ptr(g), lr, b1, b2, eps, int(t))


def calibrate(z, y, eps: float = 1e-5):
    """tau = (min positive z) - eps rounded toward -inf; returns (tau, n_positive)."""
    z = np.ascontiguousarray(z, dtype=np.float64)
    y = np.ascontiguousarray(np.asarray(y).astype(np.uint8))
    tau = np.zeros(1, dtype=np.float64)
    npos = lib().orc_calibrate(_ptr(z), _ptr(y), z.shape[0], float(eps), _ptr(tau))
    return float(tau[0]), int(npos)


def count(z, y, tau: float) -> dict:
    z = np.ascontiguousarray(z, dtype=np.float64)
    y = np.ascontiguousarray(np.asarray(y).astype(np.uint8))
    out = np.zeros(4, dtype=np.int64)
    lib().orc_count(_ptr(z), _ptr(y), z.shape[0], float(tau), _ptr(out))
    return {"FN": int(out[0]), "FP": int(out[1]), "TP": int(out[2]), "TN": int(out[3])}


ENC_W = (2, 3, 4, 6, 4, 6)


def philox4x64(counter, key) -> np.ndarray:
    """One Philox4x64-10 block (four uint64 words) for a 4-word counter and 2-word key."""
    c = np.ascontiguousarray(np.asarray(counter, dtype=np.uint64))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint64))
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_philox4x64(_ptr(c), _ptr(k), _ptr(out))
    return out


def sample(kind: int, n: int, seed: int, first: int = 0, qexp: int = 20,
           nthreads: int | None = None) -> np.ndarray:
    """Queries first .. first+n-1 of the counter-based stream (seed, kind): the
    per-iteration Uniform draw of Alg. 1, float32 [n][enc width] on the 2^-qexp grid."""
    q = np.zeros((n, ENC_W[kind]), dtype=np.float32)
    if lib().orc_sample(int(kind), int(qexp), int(seed), int(first), int(n), _ptr(q), _threads(nthreads)) != 0:
        raise ValueError("oracle sample: bad kind, qexp or range")
    return q


def benefit_break_even(t_a: float, t_b: float, p_a: float, p_b: float):
    """Eq. (Benefit), Sec. 5 (Discussion, "Tightness"): with bounding method A (query time t_a,
    fraction p_a of queries passed to the exact test) against method B (t_b, p_b),
    the total time of N queries is N t_i + p_i N t for an exact test of cost t, so A
    wins iff t_a + p_a t < t_b + p_b t.  Returns (t*, side): A wins for t > t* when
    side is '>' (p_a < p_b), for t < t* when side is '<' (p_a > p_b); t* is None
    when p_a == p_b (then A wins iff t_a < t_b)."""
    if p_a == p_b:
        return None, "<" if t_a < t_b else ">"
    t_star = (t_b - t_a) / (p_a - p_b)
    return t_star, ">" if p_a < p_b else "<"


def three_way(z_outer, tau_outer: float, z_inner, tau_inner: float) -> np.ndarray:
    """Broad-phase class of each query from a bound and an inverted bound (Sec. 4.4, the
    variant with the asymmetry weights swapped): the outer network bounds g, so
    z_outer < tau_outer means certainly outside; the inner network bounds the complement
    1 - g (the swapped-weight network with its logit negated), so z_inner < tau_inner
    means certainly inside.  Codes: 0 certainly outside, 1 certainly inside, 2 neither
    (the only queries an exact test must see).  A query that both networks call certain,
    which cannot happen on either network's calibration set, is 2."""
    z_outer = np.asarray(z_outer, dtype=np.float64)
    z_inner = np.asarray(z_inner, dtype=np.float64)
    out_ = z_outer < tau_outer
    in_ = z_inner < tau_inner
    codes = np.full(z_outer.shape[0], 2, dtype=np.uint8)
    codes[out_ & ~in_] = 0
    codes[in_ & ~out_] = 1
    return codes


ENC_PAPER_W = (2, 3, 4, 6, 6, 6)


def paper_encoding(kind: int, q) -> np.ndarray:
    """The paper's query parameterisation (Suppl. "Parameterization"), in FP64: rays as start
    and direction (unchanged), boxes as their two corners (c - e, c + e), planes as a point
    p0 on the plane and the normal; p0 = off n / |n|^2, the plane's point nearest the origin
    (n . p0 = off).  Points are unchanged."""
    q = np.asarray(q, dtype=np.float64)
    if kind == 5:  # box: centre, half-extents -> min corner, max corner
        return np.concatenate([q[:, :3] - q[:, 3:], q[:, :3] + q[:, 3:]], axis=1)
    if kind == 4:  # plane: normal, offset -> p0, normal
        nrm = q[:, :3]
        p0 = q[:, 3:4] * nrm / np.sum(nrm * nrm, axis=1, keepdims=True)
        return np.concatenate([p0, nrm], axis=1)
    return q.copy()


def canonical_ray(rays, centres, R: float = 2.0):
    """The cascade's network input for (ray, object) pairs: the ray in the object's frame
    with its origin moved to its entry point into the ball of radius R around the object's
    centre, by the library's defined FP32 operation sequence (oracle.c, orc_canonical_ray).
    rays [n][6] (origin, direction), centres [n][3] (the object of each pair).  Returns
    (q6 float32 [n][6], met bool [n]); rows that miss the ball are zero."""
    rays = np.ascontiguousarray(rays, dtype=np.float32)
    centres = np.ascontiguousarray(centres, dtype=np.float32)
    n = rays.shape[0]
    q6 = np.zeros((n, 6), dtype=np.float32)
    met = np.zeros(n, dtype=np.uint8)
    R2 = np.float32(np.float32(R) * np.float32(R))
    if lib().orc_canonical_ray(_ptr(rays), _ptr(centres), n, float(R2), _ptr(q6), _ptr(met)) != 0:
        raise ValueError("oracle canonical_ray: bad arguments")
    return q6, met.astype(bool)


def canonical_ray_f64(rays, centres, R: float = 2.0):
    """The same entry point in FP64 (smaller root of |w + s d| = R, clamped at s = 0); the
    real-valued counterpart the FP32 sequence is pinned against.  Returns (p [n][3], met)."""
    rays = np.ascontiguousarray(rays, dtype=np.float32)
    centres = np.ascontiguousarray(centres, dtype=np.float32)
    n = rays.shape[0]
    p = np.zeros((n, 3), dtype=np.float64)
    met = np.zeros(n, dtype=np.uint8)
    if lib().orc_canonical_ray_f64(_ptr(rays), _ptr(centres), n, float(R), _ptr(p), _ptr(met)) != 0:
        raise ValueError("oracle canonical_ray_f64: bad arguments")
    return p, met.astype(bool)
