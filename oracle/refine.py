"""FP64 oracle of the zeroth-order path refinement of Section III (the RRT
path smoothed by one MPPI step whose horizon is the whole plan).

TEST INFRASTRUCTURE ONLY (like the rest of this package): the tests and the
benchmark's CPU leg use it; the product library never does.  It shares no
code with the CUDA path.

The paper optimises the knots of a B-spline through the plan, minimising the
path length with a collision penalty, by one MPPI step (Section II-D).  The
readings taken here:

1. the path is the clamped uniform cubic B-spline of the control points
   P_0 .. P_{N-1} (the paper's knots): the control polygon padded with two
   more copies of each endpoint, so the curve starts at P_0 and ends at
   P_{N-1}; it has N + 1 segments, segment j using padded points j .. j + 3
   with the uniform cubic basis
     b0 = (1 - u)^3 / 6, b1 = (3u^3 - 6u^2 + 4) / 6,
     b2 = (-3u^3 + 3u^2 + 3u + 1) / 6, b3 = u^3 / 6;
2. each segment is sampled at u = m / M, m = 0 .. M - 1, and the path's last
   point P_{N-1} is added: (N + 1) M + 1 points, spheres of radius r;
3. rollout k perturbs the interior control points by eps[k] (the endpoints
   stay where they are: their perturbations are ignored);

Steps 2-3 decide the sphere centres the metric sees, so they are computed in
float32 with every operation rounded, in this order (the device repeats it):
   c = P + eps; u = m / M; u2 = u u; u3 = u2 u; v = 1 - u;
   b0 = ((v v) v) / 6, b1 = ((3 u3 - 6 u2) + 4) / 6,
   b2 = (((3 u2 - 3 u3) + 3 u) + 1) / 6, b3 = u3 / 6,
   x = ((b0 Q0 + b1 Q1) + b2 Q2) + b3 Q3;
the costs and the update are FP64;
4. cost: C^k = w_length L^k + w_collision sum over the points of the Eq. 11
   cost averaged over the neighbour set, L^k the length of the polyline
   through the points;
5. Eq. 10 weights w^k = exp(-(C^k - min C) / lambda) / sum, and the update
   P' = P + sum_k w^k eps[k] on the interior points.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import Params, group_reduce, query


@dataclass
class RefineDesc:
    K: int
    N: int
    M: int = 8
    radius: float = 0.05
    nsigma: float = 1.0
    lam: float = 1.0
    w_length: float = 1.0
    w_collision: float = 10.0


def basis(u):
    """Uniform cubic B-spline basis (4 weights) at parameter(s) u, FP64."""
    u = np.asarray(u, np.float64)
    return np.stack([(1 - u) ** 3 / 6, (3 * u ** 3 - 6 * u ** 2 + 4) / 6,
                     (-3 * u ** 3 + 3 * u ** 2 + 3 * u + 1) / 6, u ** 3 / 6], -1)


def basis32(m, M):
    """The basis at u = m / M in float32, in the stated operation order."""
    f = np.float32
    u = f(m) / f(M)
    u2 = u * u
    u3 = u2 * u
    v = f(1) - u
    return (((v * v) * v) / f(6), ((f(3) * u3 - f(6) * u2) + f(4)) / f(6),
            (((f(3) * u2 - f(3) * u3) + f(3) * u) + f(1)) / f(6), u3 / f(6))


def points(ctrl, M):
    """The (N + 1) M + 1 sample points of the clamped spline of ctrl [N,3], or
    of a batch [K,N,3] (float32 in, float32 out, the stated operation order)."""
    P = np.asarray(ctrl, np.float32)
    single = P.ndim == 2
    if single:
        P = P[None]
    Q = np.concatenate([P[:, :1], P[:, :1], P, P[:, -1:], P[:, -1:]], axis=1)
    K, N = P.shape[0], P.shape[1]
    out = np.empty((K, (N + 1) * M + 1, 3), np.float32)
    for m in range(M):
        b0, b1, b2, b3 = basis32(m, M)
        seg = ((b0 * Q[:, 0:N + 1] + b1 * Q[:, 1:N + 2]) + b2 * Q[:, 2:N + 3]) + b3 * Q[:, 3:N + 4]
        out[:, m:(N + 1) * M:M] = seg
    out[:, -1] = P[:, -1]
    return out[0] if single else out


def refine(scene, ctrl, eps, d: RefineDesc, params: Params | None = None) -> dict:
    """One refinement step: new control points, per-rollout cost and weights."""
    params = params or Params()
    ctrl32 = np.asarray(ctrl, np.float32)
    eps32 = np.array(eps, np.float32)
    eps32[:, 0, :] = 0.0
    eps32[:, -1, :] = 0.0
    pts = points(ctrl32[None] + eps32, d.M)   # [K,P,3] float32
    P = pts.shape[1]
    length = np.linalg.norm(np.diff(pts.astype(np.float64), axis=1), axis=2).sum(1)
    sph = np.c_[pts.reshape(-1, 3), np.full(d.K * P, d.radius, np.float32)].astype(np.float32)
    res = query(scene, sph, 0, d.nsigma, params)
    col, _ = group_reduce(res["mean_cost"], res["collide"], P)
    cost = d.w_length * length + d.w_collision * col
    e = np.exp(-(cost - cost.min()) / d.lam)
    w = e / e.sum()
    new = ctrl32.astype(np.float64) + np.einsum("k,knd->nd", w, eps32.astype(np.float64))
    return {"ctrl": new, "cost": cost, "weights": w, "length": length, "collision": col, "points": pts,
            "query": res}


__all__ = ["RefineDesc", "basis", "basis32", "points", "refine"]
