"""FP64 oracle of the pose chain that turns per-waypoint rigid poses into the
sphere centres the metric consumes, and its adjoint.

TEST INFRASTRUCTURE ONLY (see the package docstring).

A pose is (t, w): translation t and axis-angle rotation w (rotation vector),
R(w) = exp([w]x) (Rodrigues).  Sphere k of a waypoint sits at body-frame
offset p_k:   c_k = t + R(w) p_k.

Adjoint, for an upstream gradient g_k = dL/dc_k:
  dL/dt = sum_k g_k
  dL/dw = J_l(w)^T sum_k (R(w) p_k) x g_k
with the left Jacobian of SO(3)
  J_l(w) = I + (1 - cos th)/th^2 [w]x + (th - sin th)/th^3 [w]x^2.
(A left perturbation R(w + e) = exp([J_l e]x) R(w) moves R p by
-[R p]x J_l e, whose transpose applied to g is J_l^T ((R p) x g).)
"""
from __future__ import annotations

import numpy as np


def _skew(v):
    z = np.zeros(v.shape[:-1])
    return np.stack([
        np.stack([z, -v[..., 2], v[..., 1]], -1),
        np.stack([v[..., 2], z, -v[..., 0]], -1),
        np.stack([-v[..., 1], v[..., 0], z], -1)], -2)


def _coeffs(th):
    """sin(th)/th, (1-cos th)/th^2, (th - sin th)/th^3 with series near 0."""
    th = np.asarray(th, np.float64)
    small = th < 1e-4
    ts = np.where(small, 1.0, th)
    a = np.where(small, 1.0 - th ** 2 / 6.0, np.sin(ts) / ts)
    b = np.where(small, 0.5 - th ** 2 / 24.0, (1.0 - np.cos(ts)) / ts ** 2)
    c = np.where(small, 1.0 / 6.0 - th ** 2 / 120.0, (ts - np.sin(ts)) / ts ** 3)
    return a, b, c


def rotation(w):
    """Rodrigues: R = I + sin(th)/th [w]x + (1-cos th)/th^2 [w]x^2."""
    w = np.asarray(w, np.float64)
    th = np.linalg.norm(w, axis=-1)
    a, b, _ = _coeffs(th)
    K = _skew(w)
    eye = np.broadcast_to(np.eye(3), K.shape)
    return eye + a[..., None, None] * K + b[..., None, None] * (K @ K)


def left_jacobian(w):
    w = np.asarray(w, np.float64)
    th = np.linalg.norm(w, axis=-1)
    _, b, c = _coeffs(th)
    K = _skew(w)
    eye = np.broadcast_to(np.eye(3), K.shape)
    return eye + b[..., None, None] * K + c[..., None, None] * (K @ K)


def centres(poses, offsets):
    """poses [P,6] = (t, w); offsets [K,3] -> centres [P,K,3]."""
    poses = np.asarray(poses, np.float64)
    offsets = np.asarray(offsets, np.float64)
    R = rotation(poses[:, 3:])
    return poses[:, None, :3] + np.einsum("pab,kb->pka", R, offsets)


def pose_grad(poses, offsets, grad_centres):
    """Adjoint of centres(): grad_centres [P,K,3] -> grad_poses [P,6]."""
    poses = np.asarray(poses, np.float64)
    offsets = np.asarray(offsets, np.float64)
    g = np.asarray(grad_centres, np.float64)
    R = rotation(poses[:, 3:])
    Rp = np.einsum("pab,kb->pka", R, offsets)
    gt = g.sum(axis=1)
    torque = np.cross(Rp, g).sum(axis=1)
    Jl = left_jacobian(poses[:, 3:])
    gw = np.einsum("pba,pb->pa", Jl, torque)
    return np.concatenate([gt, gw], axis=1)
