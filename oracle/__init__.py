"""FP64 CPU oracle for the CollisionSplatting conservative metric.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark import this package; the product library never does.  It
shares no code with the CUDA path.

The arithmetic lives in ``cs_oracle.c`` (brute force over every pair, double
precision, paper Section II, Eq. 2 and Eq. 5-8, Eq. 11).  This module only
compiles it with gcc, marshals arrays through ctypes and applies the group
sums of Section II-D (sum over links and horizon) with numpy.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cs_oracle.c")
_LIB = os.path.join(_HERE, "libcs_oracle.so")

MODE_MEAN, MODE_SUM, MODE_MIN, MODE_SOFTMIN = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math: IEEE double throughout).

    CS_ORACLE_LIB may name another build of the same source (the mutation
    tests plant a mistake in a copy and check that the pins catch it)."""
    override = os.environ.get("CS_ORACLE_LIB")
    if override:
        return override
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("gamma", ctypes.c_double),
        ("d_max", ctypes.c_double),
        ("s_min", ctypes.c_double),
        ("eps", ctypes.c_double),
        ("tau", ctypes.c_double),
        ("k_thr", ctypes.c_int64),
        ("opacity_min", ctypes.c_double),
        ("extent_max", ctypes.c_double),
        ("use_filter", ctypes.c_int32),
        ("nthreads", ctypes.c_int32),
        ("band", ctypes.c_double),
        ("exact_variance", ctypes.c_int32),
    ]


class _Outputs(ctypes.Structure):
    _fields_ = [(name, ctypes.c_void_p) for name in (
        "sum_cost", "mean_cost", "count_nbr", "count_in", "collide", "min_s2", "softmin",
        "band_cut", "band_in", "cond", "min_cond", "band_kink", "cond_cost")]


@dataclass
class Params:
    """Metric parameters (paper Eq. 11, Section II-C/E); defaults are the
    readings used throughout: gamma=5, d_max=1, s_min=1, eps=1e-6, tau=0.05,
    k_thr=0, floater filter (opacity < 0.05 and max scale > 0.1)."""
    gamma: float = 5.0
    d_max: float = 1.0
    s_min: float = 1.0
    eps: float = 1e-6
    tau: float = 0.05
    k_thr: int = 0
    opacity_min: float = 0.05
    extent_max: float = 0.1
    use_filter: bool = True
    nthreads: int = 0
    band: float = 1e-5  # width of the reporting bands (band_cut, band_in, band_kink)
    exact_variance: bool = False  # the exact variance of Eq. 5 instead of Eq. 7's linearisation

    @property
    def s_cut(self) -> float:
        return self.s_min + np.log(1.0 / self.eps) / self.gamma

    def _c(self) -> _Params:
        return _Params(self.gamma, self.d_max, self.s_min, self.eps, self.tau, int(self.k_thr),
                       self.opacity_min, self.extent_max, int(bool(self.use_filter)),
                       int(self.nthreads), float(self.band), int(bool(self.exact_variance)))


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.orc_query.argtypes = [ctypes.c_int64, P, P, P, P, ctypes.c_int, P, ctypes.c_int64, P,
                                  ctypes.POINTER(_Params), ctypes.POINTER(_Outputs)]
        lib.orc_grad.argtypes = [ctypes.c_int64, P, P, P, P, ctypes.c_int, P, ctypes.c_int64, P,
                                 ctypes.POINTER(_Params), ctypes.c_int, P, P, P]
        lib.orc_pair.argtypes = [P, P, P, ctypes.c_int, P, ctypes.c_double,
                                 ctypes.POINTER(_Params), P]
        lib.orc_covariances.argtypes = [ctypes.c_int64, P, P, P, ctypes.POINTER(_Params), P, P]
        lib.orc_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _f32(a, cols=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    if cols is not None:
        a = a.reshape(-1, cols)
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data


def _scene_arrays(scene):
    means = _f32(scene["means"], 3)
    scales = _f32(scene["scales"], 3)
    quats = _f32(scene["quats"], 4)
    op = scene.get("opacity")
    op = None if op is None else _f32(op).reshape(-1)
    return means, scales, quats, op


def _nsigma_array(nsigma, Q):
    ns = np.asarray(nsigma, dtype=np.float64)
    if ns.ndim == 0:
        ns = np.full(Q, float(ns))
    return np.ascontiguousarray(ns.reshape(Q))


def num_threads() -> int:
    return int(_load().orc_num_threads())


def query(scene, prims, prim_type: int, nsigma, params: Params | None = None) -> dict:
    """Every per-query output of the metric for Q primitives.

    scene: dict with means [N,3], scales [N,3], quats [N,4] (w,x,y,z), opacity [N].
    prims: [Q,4] spheres (c, r) for prim_type 0, [Q,10] ellipsoids
    (c, q wxyz, a, b, c) for prim_type 1.  nsigma: scalar or [Q].
    """
    params = params or Params()
    lib = _load()
    means, scales, quats, op = _scene_arrays(scene)
    prims = _f32(prims, 4 if prim_type == 0 else 10)
    Q = prims.shape[0]
    ns = _nsigma_array(nsigma, Q)
    res = {
        "sum_cost": np.zeros(Q), "mean_cost": np.zeros(Q),
        "count_nbr": np.zeros(Q, np.int64), "count_in": np.zeros(Q, np.int64),
        "collide": np.zeros(Q, np.uint8), "min_s2": np.zeros(Q), "softmin": np.zeros(Q),
        "band_cut": np.zeros(Q, np.int64), "band_in": np.zeros(Q, np.int64),
        "cond": np.zeros(Q), "min_cond": np.zeros(Q), "band_kink": np.zeros(Q, np.int64),
        "cond_cost": np.zeros(Q),
    }
    outs = _Outputs(*[res[k].ctypes.data for k, _ in _Outputs._fields_])
    rc = lib.orc_query(means.shape[0], _ptr(means), _ptr(scales), _ptr(quats), _ptr(op), prim_type,
                       _ptr(prims), Q, _ptr(ns), ctypes.byref(params._c()), ctypes.byref(outs))
    if rc != 0:
        raise ValueError(f"oracle query failed ({rc}): invalid primitive")
    return res


def metric(res: dict, mode: int) -> np.ndarray:
    """The per-query metric selected by mode (Section II-B/D readings)."""
    return {MODE_MEAN: res["mean_cost"], MODE_SUM: res["sum_cost"],
            MODE_MIN: res["min_s2"], MODE_SOFTMIN: res["softmin"]}[mode]


def grad(scene, prims, prim_type: int, nsigma, mode: int = MODE_MEAN,
         grad_out=None, params: Params | None = None, return_scale: bool = False):
    """Analytic gradient of the per-query metric with respect to the
    primitive centres, [Q,3], scaled by grad_out [Q] (ones if None).  With
    return_scale, also the sum of the norms of the summed terms per query
    (each term's size counted as the sum of the sizes of its two parts, which
    may cancel: the conditioning of the sum)."""
    params = params or Params()
    lib = _load()
    means, scales, quats, op = _scene_arrays(scene)
    prims = _f32(prims, 4 if prim_type == 0 else 10)
    Q = prims.shape[0]
    ns = _nsigma_array(nsigma, Q)
    go = None if grad_out is None else np.ascontiguousarray(np.asarray(grad_out, np.float64).reshape(Q))
    g = np.zeros((Q, 3))
    sc = np.zeros(Q)
    rc = lib.orc_grad(means.shape[0], _ptr(means), _ptr(scales), _ptr(quats), _ptr(op), prim_type,
                      _ptr(prims), Q, _ptr(ns), ctypes.byref(params._c()), mode, _ptr(go), _ptr(g),
                      _ptr(sc))
    if rc != 0:
        raise ValueError(f"oracle grad failed ({rc}): invalid primitive")
    return (g, sc) if return_scale else g


def pair(mean, scale, quat, prim, prim_type: int, nsigma: float,
         params: Params | None = None) -> dict:
    """Terms of one pair: s2 (Eq. 5), var (Eq. 7), st2 (Eq. 8), dc (Eq. 11), raw."""
    params = params or Params()
    lib = _load()
    m, s, q = _f32(mean), _f32(scale), _f32(quat)
    p = _f32(prim)
    out = np.zeros(5)
    rc = lib.orc_pair(_ptr(m), _ptr(s), _ptr(q), prim_type, _ptr(p), float(nsigma),
                      ctypes.byref(params._c()), _ptr(out))
    if rc != 0:
        raise ValueError("invalid primitive")
    return dict(zip(("s2", "var", "st2", "dc", "raw"), out.tolist()))


def covariances(scene, params: Params | None = None):
    """Eq. 2 covariance [N,3,3] of every Gaussian and the floater-filter mask."""
    params = params or Params()
    lib = _load()
    means, scales, quats, op = _scene_arrays(scene)
    n = scales.shape[0]
    sig = np.zeros((n, 3, 3))
    keep = np.zeros(n, np.uint8)
    lib.orc_covariances(n, _ptr(scales), _ptr(quats), _ptr(op), ctypes.byref(params._c()),
                        _ptr(sig), _ptr(keep))
    return sig, keep.astype(bool)


def group_reduce(per_query_metric, per_query_collide, group_size: int):
    """Section II-D/E group outputs: the metric summed over each run of
    group_size consecutive queries (links, then horizon steps) and the
    collision flag OR-ed over it (an edge collides if any point does).  The
    last group may be shorter."""
    m = np.asarray(per_query_metric, np.float64)
    c = np.asarray(per_query_collide).astype(bool)
    Q = m.shape[0]
    ng = (Q + group_size - 1) // group_size
    gm = np.array([m[g * group_size:(g + 1) * group_size].sum() for g in range(ng)])
    gc = np.array([c[g * group_size:(g + 1) * group_size].any() for g in range(ng)], np.uint8)
    return gm, gc
