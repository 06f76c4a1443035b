"""B300 engine for the CollisionSplatting conservative collision metric
(arXiv 2609.35619, Section II-B/D/E) behind a C ABI (include/cs_b300.h).

Python surface (argument marshalling over the C entry points; every step of
the metric runs in the library's CUDA kernels):

  Scene(means, scales, quats, opacity, ...)    cs_scene_create / destroy
  Scene.query(prims, nsigma, ...)              cs_query
  Scene.query_grad(prims, nsigma, ...)         cs_query_grad
  pose_spheres / pose_spheres_grad             cs_pose_spheres(_grad)
  CollisionCost.apply(poses, ...)              torch.autograd.Function over the
                                               pose chain and the metric
The raw one-to-one binding is `paper_2609_35619_b300.abi`.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

from . import abi
from .abi import (CS_METRIC_MEAN_COST, CS_METRIC_MIN_S2, CS_METRIC_SOFTMIN_S2, CS_METRIC_SUM_COST,
                  CS_PRIM_ELLIPSOID, CS_PRIM_SPHERE, CsError, check)

__all__ = ["Scene", "QueryParams", "pose_spheres", "pose_spheres_grad", "CollisionCost", "abi",
           "CS_PRIM_SPHERE", "CS_PRIM_ELLIPSOID", "CS_METRIC_MEAN_COST", "CS_METRIC_SUM_COST",
           "CS_METRIC_MIN_S2", "CS_METRIC_SOFTMIN_S2", "CsError"]


@dataclass
class QueryParams:
    """Per-call parameters (cs_params); defaults are the library's."""
    gamma: float = 5.0
    d_max: float = 1.0
    s_min: float = 1.0
    eps: float = 1e-6
    tau: float = 0.05
    k_thr: int = 0
    mode: int = CS_METRIC_MEAN_COST
    group_size: int = 0
    tile_config: int = 0

    def to_c(self) -> abi.cs_params:
        p = abi.cs_params()
        check(abi.cs_params_init(p))
        p.gamma, p.d_max, p.s_min, p.eps, p.tau = self.gamma, self.d_max, self.s_min, self.eps, self.tau
        p.k_thr, p.mode, p.group_size, p.tile_config = self.k_thr, self.mode, self.group_size, self.tile_config
        return p


def _torch():
    import torch
    return torch


def _as_f32(t, device):
    torch = _torch()
    if not isinstance(t, torch.Tensor):
        t = torch.as_tensor(t)
    return t.to(device=device, dtype=torch.float32).contiguous()


class Scene:
    """A resident scene on the current CUDA device (cs_scene_create)."""

    def __init__(self, means, scales, quats, opacity=None, *, use_filter=True, opacity_min=0.05,
                 extent_max=0.1, cell_size=0.0, tier_quantile=0.0, device="cuda", stream=None):
        torch = _torch()
        dev = torch.device(device)
        m = _as_f32(means, dev).reshape(-1, 3)
        s = _as_f32(scales, dev).reshape(-1, 3)
        q = _as_f32(quats, dev).reshape(-1, 4)
        o = None if opacity is None else _as_f32(opacity, dev).reshape(-1)
        d = abi.cs_scene_desc()
        d.n = m.shape[0]
        d.means, d.scales, d.quats = abi.ptr(m), abi.ptr(s), abi.ptr(q)
        d.opacity = abi.ptr(o)
        d.on_device = 1 if dev.type == "cuda" else 0
        d.use_filter = int(bool(use_filter))
        d.opacity_min, d.extent_max = opacity_min, extent_max
        d.cell_size, d.tier_quantile = cell_size, tier_quantile
        self._h = ctypes.c_void_p()
        check(abi.cs_scene_create(d, stream, self._h))
        self.device = dev

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            check(abi.cs_scene_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        inf = abi.cs_scene_info()
        check(abi.cs_scene_info_get(self._h, inf))
        return {"n_input": inf.n_input, "n_kept": inf.n_kept, "n_grid": inf.n_grid,
                "n_large": inf.n_large, "n_invalid": inf.n_invalid, "dims": list(inf.dims),
                "cell_size": inf.cell_size, "sigma_tier": inf.sigma_tier, "lo": list(inf.lo),
                "hi": list(inf.hi), "device_bytes": inf.device_bytes}

    def export(self, stream=None):
        torch = _torch()
        n = self.info()["n_kept"]
        pos = torch.empty((n, 4), dtype=torch.float32, device=self.device)
        cov = torch.empty((n, 8), dtype=torch.float32, device=self.device)
        idx = torch.empty((n,), dtype=torch.int32, device=self.device)
        check(abi.cs_scene_export(self._h, pos, cov, idx, stream))
        return pos, cov, idx

    def query(self, prims, nsigma=1.0, *, prim_type=CS_PRIM_SPHERE, params: QueryParams | None = None,
              nsigma_per_query=None, want_count=False, pair_stats=None, stream=None,
              eval_events=None, out=None, kernel_stats=None) -> dict:
        """cs_query on device tensors; returns a dict of device tensors."""
        torch = _torch()
        params = params or QueryParams()
        cols = 4 if prim_type == CS_PRIM_SPHERE else 10
        prims = _as_f32(prims, self.device).reshape(-1, cols)
        Q = prims.shape[0]
        if out is None:
            out = {"metric": torch.empty(Q, dtype=torch.float32, device=self.device),
                   "collide": torch.empty(Q, dtype=torch.uint8, device=self.device)}
        p = params.to_c()
        _set_events(p, eval_events)
        p.stream = abi.stream_handle(stream)
        if nsigma_per_query is not None:
            nsq = _as_f32(nsigma_per_query, self.device).reshape(Q)
            out["_ns"] = nsq
            p.nsigma_per_query = abi.ptr(nsq)
        if want_count:
            if "count" not in out:
                out["count"] = torch.empty(Q, dtype=torch.int32, device=self.device)
            p.out_count = abi.ptr(out["count"])
        if params.group_size > 0:
            ng = (Q + params.group_size - 1) // params.group_size
            if "group_metric" not in out:
                out["group_metric"] = torch.empty(ng, dtype=torch.float32, device=self.device)
                out["group_collide"] = torch.empty(ng, dtype=torch.uint8, device=self.device)
            p.out_group_metric = abi.ptr(out["group_metric"])
            p.out_group_collide = abi.ptr(out["group_collide"])
        if pair_stats is not None:
            p.out_pair_stats = abi.ptr(pair_stats)
        if kernel_stats is not None:
            p.out_kernel_stats = abi.ptr(kernel_stats)
        check(abi.cs_query(self._h, prim_type, prims, Q, float(nsigma), out["metric"], out["collide"], p))
        out.pop("_ns", None)
        return out

    def query_grad(self, prims, nsigma=1.0, *, grad_out=None, prim_type=CS_PRIM_SPHERE,
                   params: QueryParams | None = None, nsigma_per_query=None, stream=None,
                   eval_events=None, out=None):
        """cs_query_grad: d metric / d centre, [Q,3] device tensor."""
        torch = _torch()
        params = params or QueryParams()
        cols = 4 if prim_type == CS_PRIM_SPHERE else 10
        prims = _as_f32(prims, self.device).reshape(-1, cols)
        Q = prims.shape[0]
        g = out if out is not None else torch.empty((Q, 3), dtype=torch.float32, device=self.device)
        p = params.to_c()
        p.stream = abi.stream_handle(stream)
        _set_events(p, eval_events)
        keep = []
        if nsigma_per_query is not None:
            nsq = _as_f32(nsigma_per_query, self.device).reshape(Q)
            keep.append(nsq)
            p.nsigma_per_query = abi.ptr(nsq)
        go = None if grad_out is None else _as_f32(grad_out, self.device).reshape(-1)
        check(abi.cs_query_grad(self._h, prim_type, prims, Q, float(nsigma), go, g, p))
        return g

    def sync(self, stream=None):
        check(abi.cs_sync(self._h, stream))


def _set_events(p, events):
    """Record a (start, stop) pair of torch.cuda.Event around the fused kernel."""
    if events is None:
        return
    for k, ev in enumerate(events):
        if not ev.cuda_event:  # torch creates the event lazily on first record
            ev.record()
        p.eval_events[k] = ev.cuda_event


def pose_spheres(poses, offsets, radius: float, stream=None):
    """cs_pose_spheres: poses [P,6] (t, axis-angle), offsets [K,3] -> [P*K,4]."""
    torch = _torch()
    poses = poses.contiguous()
    offsets = offsets.contiguous()
    P, K = poses.shape[0], offsets.shape[0]
    out = torch.empty((P * K, 4), dtype=torch.float32, device=poses.device)
    check(abi.cs_pose_spheres(poses, P, offsets, K, radius, out, stream))
    return out


def pose_spheres_grad(poses, offsets, grad_centres, stream=None):
    torch = _torch()
    poses = poses.contiguous()
    offsets = offsets.contiguous()
    P, K = poses.shape[0], offsets.shape[0]
    g = torch.empty((P, 6), dtype=torch.float32, device=poses.device)
    check(abi.cs_pose_spheres_grad(poses, P, offsets, K, grad_centres.contiguous(), g, stream))
    return g


def _make_autograd():
    torch = _torch()

    class CollisionCost(torch.autograd.Function):
        """Per-pose collision cost: the metric of the K body spheres of each
        pose summed over the spheres (Section II-D sums over links), with the
        gradient through cs_query_grad and the pose-chain adjoint.

        forward(poses [P,6], scene, offsets [K,3], radius, nsigma, params) -> [P]
        """

        @staticmethod
        def forward(ctx, poses, scene, offsets, radius, nsigma, params=None):
            params = params or QueryParams()
            K = offsets.shape[0]
            spheres = pose_spheres(poses.detach().float(), offsets.float(), radius)
            qp = QueryParams(**{**params.__dict__, "group_size": K})
            out = scene.query(spheres, nsigma, params=qp)
            ctx.save_for_backward(poses, offsets, spheres)
            ctx.scene, ctx.nsigma, ctx.qp = scene, nsigma, qp
            return out["group_metric"]

        @staticmethod
        def backward(ctx, grad_pose_cost):
            poses, offsets, spheres = ctx.saved_tensors
            gc = ctx.scene.query_grad(spheres, ctx.nsigma, grad_out=grad_pose_cost.float().contiguous(),
                                      params=ctx.qp)
            gp = pose_spheres_grad(poses.detach().float(), offsets.float(), gc)
            return gp.to(poses.dtype), None, None, None, None, None

    return CollisionCost


class _Lazy:
    _cls = None

    def __getattr__(self, name):
        if _Lazy._cls is None:
            _Lazy._cls = _make_autograd()
        return getattr(_Lazy._cls, name)


CollisionCost = _Lazy()
