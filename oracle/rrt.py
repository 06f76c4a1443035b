"""Oracle of one batched RRT extension with the collision rule of Section II-E.

TEST INFRASTRUCTURE ONLY (like the rest of this package): the tests and the
benchmark's CPU leg use it; the product library never does.  It shares no
code with the CUDA path.

The paper grows its tree 32 nodes at a time and checks every candidate edge
with the metric (a state collides when a link has more than k_thr Gaussians
with st^2 < 1).  For a robot that is one sphere of radius r, one extension
with B samples s_b takes these steps:

1. nearest: n_b = the tree node closest to s_b (squared Euclidean distance,
   the lowest index on ties);
2. steer: d = s_b - x[n_b], L = |d|; the new node is s_b when L <= step,
   else x[n_b] + d * (step / L);
3. edge: M points along the edge, p_m = x[n_b] + (new - x[n_b]) * (m + 1) / M
   for m < M - 1, and p_{M-1} = new;
4. check: the edge collides when any of its points does (Section II-E);
5. insert: the new nodes of the free edges are appended in sample order
   (node count + rank among the free edges), with parent n_b, while the
   capacity lasts.

Steps 1-3 decide integers and positions, so they are computed in FP32 with
the operations in a fixed order (no fused multiply-add), the precision the
device path uses; step 4 uses the FP64 metric of this package.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import Params, group_reduce, query


@dataclass
class RrtDesc:
    B: int = 32
    M: int = 16
    step: float = 0.5
    radius: float = 0.15
    nsigma: float = 1.0
    capacity: int = 1 << 16


def _f(x):
    return np.float32(x)


def nearest(nodes, count, samples):
    """Index of the closest of nodes[:count] to each sample (FP32, ties -> lowest)."""
    nd = np.asarray(nodes, np.float32)[:count]
    out = np.empty(len(samples), np.int64)
    for b, s in enumerate(np.asarray(samples, np.float32)):
        dx, dy, dz = nd[:, 0] - s[0], nd[:, 1] - s[1], nd[:, 2] - s[2]
        d2 = (dx * dx + dy * dy) + dz * dz  # float32 throughout, this order
        out[b] = int(np.argmin(d2))         # first index of the minimum
    return out


def steer(x_near, sample, step):
    """New node of one edge (FP32)."""
    x_near = np.asarray(x_near, np.float32)
    s = np.asarray(sample, np.float32)
    d = s - x_near
    L = np.sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2], dtype=np.float32)
    if L <= _f(step):
        return s.copy()
    f = _f(step) / L
    return x_near + d * f


def edge_points(x_near, new, M):
    """The M checked points of an edge (FP32); the last one is the new node."""
    x_near = np.asarray(x_near, np.float32)
    new = np.asarray(new, np.float32)
    dd = new - x_near
    pts = np.empty((M, 3), np.float32)
    for m in range(M - 1):
        t = _f(m + 1) / _f(M)
        pts[m] = x_near + dd * t
    pts[M - 1] = new
    return pts


def extend(scene, nodes, parent, count, samples, d: RrtDesc, params: Params | None = None) -> dict:
    """One extension: nearest, steered new nodes, edge flags and the grown tree."""
    params = params or Params()
    nodes = np.array(nodes, np.float32)
    parent = np.array(parent, np.int64)
    samples = np.asarray(samples, np.float32)
    B = samples.shape[0]
    near = nearest(nodes, count, samples)
    new = np.stack([steer(nodes[near[b]], samples[b], d.step) for b in range(B)])
    pts = np.concatenate([edge_points(nodes[near[b]], new[b], d.M) for b in range(B)])
    res = query(scene, np.c_[pts, np.full(len(pts), d.radius, np.float32)], 0, d.nsigma, params)
    _, collide = group_reduce(res["mean_cost"], res["collide"], d.M)
    band = group_reduce(res["mean_cost"], res["band_in"] > 0, d.M)[1].astype(bool)
    free = collide == 0
    n = count
    for b in range(B):
        if free[b] and n < d.capacity:
            nodes[n] = new[b]
            parent[n] = near[b]
            n += 1
    return {"nearest": near, "new": new, "points": pts, "edge_collide": collide, "edge_band": band,
            "nodes": nodes, "parent": parent, "count": n}


__all__ = ["RrtDesc", "nearest", "steer", "edge_points", "extend"]
