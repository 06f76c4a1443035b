"""Oracle of the 3DGS image synthesis (Section II-A, Eq. 3-4): FP64, one pixel
at a time over every Gaussian of the scene, in ``raster.c``.

TEST INFRASTRUCTURE ONLY (like the rest of this package): the tests and the
benchmark's CPU leg use it; the product library never does.  It shares no
code with the CUDA path.  The readings of the paper it takes are listed at
the top of ``raster.c``.

Cameras are float32 rows of 16: the world-to-camera rotation R (row-major),
the translation t (x_c = R x_w + t), then fx, fy, cx, cy in pixels.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from . import Params, covariances

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "raster.c")
_LIB = os.path.join(_HERE, "libcs_oracle_raster.so")
_lib = None


class _RDesc(ctypes.Structure):
    _fields_ = [
        ("width", ctypes.c_int32),
        ("height", ctypes.c_int32),
        ("near_plane", ctypes.c_double),
        ("dilation", ctypes.c_double),
        ("bg", ctypes.c_double * 3),
        ("band_rel", ctypes.c_double),
        ("band_cond", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile raster.c with gcc (IEEE double, no contraction of float
    operations).  CS_ORACLE_RASTER_LIB may name another build of the same
    source (the mutation tests plant a mistake in a copy)."""
    override = os.environ.get("CS_ORACLE_RASTER_LIB")
    if override:
        return override
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-std=c99",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.orc_render_pixels.restype = ctypes.c_int
        lib.orc_render_pixels.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                          ctypes.POINTER(_RDesc), ctypes.c_int64, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def render(scene, colors, cams, width: int, height: int, *, near_plane: float = 0.01, dilation: float = 0.3,
           background=(0.0, 0.0, 0.0), pixels=None, use_filter: bool = True, band_rel: float = 1e-6,
           band_cond: float = 16.0) -> dict:
    """Render the pixels (view, x, y) listed in `pixels` ([P,3] int), or every
    pixel of every view when None (outputs then shaped [V,H,W,...]).

    The scene's Gaussians pass the floater filter of Section II-C first (as
    the device scene does when built with use_filter); opacity defaults to 1.
    Returns rgb, depth, alpha, ncontrib, flags, cond and slack (see raster.c)."""
    lib = _load()
    means = np.ascontiguousarray(scene["means"], np.float32).reshape(-1, 3)
    op = scene.get("opacity")
    n = means.shape[0]
    op = np.ones(n) if op is None else np.asarray(op, np.float64).reshape(-1)
    sig, keep = covariances(scene, Params(use_filter=use_filter))
    if not use_filter:
        keep = np.ones(n, bool)
    means_k = np.ascontiguousarray(means[keep])
    sig_k = np.ascontiguousarray(sig[keep].reshape(-1, 9))
    op_k = np.ascontiguousarray(op[keep])
    col_k = np.ascontiguousarray(np.asarray(colors, np.float64).reshape(-1, 3)[keep])
    cams = np.ascontiguousarray(cams, np.float32).reshape(-1, 16)
    V = cams.shape[0]
    full = pixels is None
    if full:
        v, y, x = np.meshgrid(np.arange(V), np.arange(height), np.arange(width), indexing="ij")
        pixels = np.stack([v.ravel(), x.ravel(), y.ravel()], 1)
    pixels = np.ascontiguousarray(pixels, np.int32).reshape(-1, 3)
    P = pixels.shape[0]
    d = _RDesc(width, height, near_plane, dilation, (ctypes.c_double * 3)(*background), band_rel, band_cond)
    rgb = np.zeros((P, 3))
    depth = np.zeros(P)
    alpha = np.zeros(P)
    ncontrib = np.zeros(P, np.int32)
    flags = np.zeros(P, np.int32)
    cond = np.zeros(P)
    slack = np.zeros(P)
    rc = lib.orc_render_pixels(means_k.shape[0], _p(means_k), _p(sig_k), _p(op_k), _p(col_k), V, _p(cams),
                               ctypes.byref(d), P, _p(pixels), _p(rgb), _p(depth), _p(alpha), _p(ncontrib),
                               _p(flags), _p(cond), _p(slack))
    if rc != 0:
        raise MemoryError("oracle render: allocation failed")
    out = {"rgb": rgb, "depth": depth, "alpha": alpha, "ncontrib": ncontrib, "flags": flags, "cond": cond,
           "slack": slack}
    if full:
        out = {k: a.reshape((V, height, width) + a.shape[1:]) for k, a in out.items()}
    return out


__all__ = ["render", "build"]
