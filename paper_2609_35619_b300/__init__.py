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
  Scene.autotune(prims, nsigma, ...)           cs_autotune (tile shape per batch class)
  QueryGraph(scene, prims, ...)                cs_graph_create / launch / destroy
  Server(scenes, ...)                          cs_server_* (continuous batching)
  mppi_step(scene, x0, U, eps, ...)            cs_mppi_step (one fused MPPI iteration)
  MppiGraph(scene, x0, U, eps, ...)            cs_mppi_graph_create (the iteration as a CUDA graph)
  RrtTree(scene, root, ...).extend(samples)    cs_rrt_extend (batched RRT, tree on the device)
The raw one-to-one binding is `paper_2609_35619_b300.abi`.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

from . import abi
from .abi import (CS_METRIC_FLAGS, CS_METRIC_MEAN_COST, CS_METRIC_MIN_S2, CS_METRIC_SOFTMIN_S2, CS_METRIC_SUM_COST,
                  CS_PRIM_ELLIPSOID, CS_PRIM_SPHERE, CsError, check)

__all__ = ["Scene", "QueryParams", "QueryGraph", "Server", "mppi_step", "MppiGraph", "RrtTree", "RrtGraph", "path_refine", "pose_spheres", "pose_spheres_grad", "CollisionCost", "abi",
           "CS_PRIM_SPHERE", "CS_PRIM_ELLIPSOID", "CS_METRIC_MEAN_COST", "CS_METRIC_SUM_COST",
           "CS_METRIC_MIN_S2", "CS_METRIC_SOFTMIN_S2", "CS_METRIC_FLAGS", "CsError"]


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
    exact_variance: bool = False
    sweep: tuple = ()  # n_sigma values of a conservatism sweep in one launch (2 .. 8 of them)

    def to_c(self) -> abi.cs_params:
        p = abi.cs_params()
        check(abi.cs_params_init(p))
        p.gamma, p.d_max, p.s_min, p.eps, p.tau = self.gamma, self.d_max, self.s_min, self.eps, self.tau
        p.k_thr, p.mode, p.group_size, p.tile_config = self.k_thr, self.mode, self.group_size, self.tile_config
        p.exact_variance = 1 if self.exact_variance else 0
        if len(self.sweep) > 8:
            raise ValueError("a sweep takes at most 8 n_sigma values")
        p.sweep_count = len(self.sweep) if len(self.sweep) >= 2 else 0
        for k, v in enumerate(self.sweep):
            p.sweep_nsigma[k] = float(v)
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

    def save(self, path, stream=None):
        """Write the built scene to a file (cs_scene_save)."""
        check(abi.cs_scene_save(self._h, os.fspath(path), stream))

    @classmethod
    def load(cls, path, *, device="cuda", stream=None) -> "Scene":
        """A scene read from a file of save() on the current device, without a rebuild (cs_scene_load)."""
        torch = _torch()
        self = cls.__new__(cls)
        self._h = ctypes.c_void_p()
        check(abi.cs_scene_load(os.fspath(path), stream, self._h))
        self.device = torch.device(device)
        return self

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
        S = len(params.sweep) if len(params.sweep) >= 2 else 1  # outputs: S blocks of Q rows
        if out is None:
            out = {"metric": torch.empty(S * Q, dtype=torch.float32, device=self.device),
                   "collide": torch.empty(S * Q, dtype=torch.uint8, device=self.device)}
        p = params.to_c()
        _set_events(p, eval_events)
        p.stream = abi.stream_handle(stream)
        if nsigma_per_query is not None:
            nsq = _as_f32(nsigma_per_query, self.device).reshape(Q)
            out["_ns"] = nsq
            p.nsigma_per_query = abi.ptr(nsq)
        if want_count:
            if "count" not in out:
                out["count"] = torch.empty(S * Q, dtype=torch.int32, device=self.device)
            p.out_count = abi.ptr(out["count"])
        if params.group_size > 0:
            ng = S * ((Q + params.group_size - 1) // params.group_size)
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

    def query_fwd_grad(self, prims, nsigma=1.0, *, grad_out=None, params: QueryParams | None = None,
                       nsigma_per_query=None, want_count=False, pair_stats=None, stream=None, eval_events=None,
                       out=None) -> dict:
        """cs_query_fwd_grad: the forward outputs of query() (spheres, mean or
        sum cost) and d metric / d centre ("grad", [Q,3]) from one fused
        launch; returns a dict of device tensors."""
        torch = _torch()
        params = params or QueryParams()
        prims = _as_f32(prims, self.device).reshape(-1, 4)
        Q = prims.shape[0]
        if out is None:
            out = {"metric": torch.empty(Q, dtype=torch.float32, device=self.device),
                   "collide": torch.empty(Q, dtype=torch.uint8, device=self.device)}
        if "grad" not in out:
            out["grad"] = torch.empty((Q, 3), dtype=torch.float32, device=self.device)
        p = params.to_c()
        _set_events(p, eval_events)
        p.stream = abi.stream_handle(stream)
        keep = []
        if nsigma_per_query is not None:
            nsq = _as_f32(nsigma_per_query, self.device).reshape(Q)
            keep.append(nsq)
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
        go = None if grad_out is None else _as_f32(grad_out, self.device).reshape(-1)
        check(abi.cs_query_fwd_grad(self._h, CS_PRIM_SPHERE, prims, Q, float(nsigma), go, out["metric"],
                                    out["collide"], out["grad"], p))
        return out

    def sync(self, stream=None):
        check(abi.cs_sync(self._h, stream))

    def set_appearance(self, opacity=None, colors=None, *, stream=None):
        """cs_scene_set_appearance: per input row its opacity ([n], default 1)
        and RGB colour ([n,3], default white), used by render()."""
        o = None if opacity is None else _as_f32(opacity, self.device).reshape(-1)
        c = None if colors is None else _as_f32(colors, self.device).reshape(-1, 3)
        check(abi.cs_scene_set_appearance(self._h, o, c, 1 if self.device.type == "cuda" else 0, stream))

    def render(self, cams, width: int, height: int, *, near_plane: float = 0.01, dilation: float = 0.3,
               background=(0.0, 0.0, 0.0), want_depth: bool = True, want_alpha: bool = True, stream=None,
               out=None) -> dict:
        """cs_render (Section II-A, Eq. 3-4): images of the scene from the
        cameras ([V,16] float32 rows: world-to-camera R row-major, t, fx, fy,
        cx, cy).  Returns device tensors rgb [V,H,W,3] and, if wanted, depth
        and alpha [V,H,W]."""
        torch = _torch()
        cams = _as_f32(cams, self.device).reshape(-1, 16)
        V = cams.shape[0]
        if out is None:
            out = {"rgb": torch.empty((V, height, width, 3), dtype=torch.float32, device=self.device)}
            if want_depth:
                out["depth"] = torch.empty((V, height, width), dtype=torch.float32, device=self.device)
            if want_alpha:
                out["alpha"] = torch.empty((V, height, width), dtype=torch.float32, device=self.device)
        d = abi.cs_render_desc()
        check(abi.cs_render_desc_init(d))
        d.n_views, d.width, d.height = V, int(width), int(height)
        d.near_plane, d.dilation = float(near_plane), float(dilation)
        for k in range(3):
            d.background[k] = float(background[k])
        d.stream = abi.stream_handle(stream)
        n_inst = ctypes.c_int64(0)
        d.out_instances = ctypes.pointer(n_inst)
        check(abi.cs_render(self._h, d, cams, out["rgb"], out.get("depth"), out.get("alpha")))
        self.last_render_instances = int(n_inst.value)
        return out

    def autotune(self, prims, nsigma=1.0, *, prim_type=CS_PRIM_SPHERE, params: QueryParams | None = None,
                 reps: int = 3, stream=None):
        """cs_autotune on a device batch: returns (best tile id, {id: ms})."""
        params = params or QueryParams()
        cols = 4 if prim_type == CS_PRIM_SPHERE else 10
        prims = _as_f32(prims, self.device).reshape(-1, cols)
        p = params.to_c()
        p.stream = abi.stream_handle(stream)
        ids = abi.cs_tile_configs()
        ms = (ctypes.c_float * len(ids))()
        best = ctypes.c_int32()
        check(abi.cs_autotune(self._h, prim_type, prims, prims.shape[0], float(nsigma), p, reps, best,
                              ctypes.addressof(ms), len(ids)))
        return best.value, dict(zip(ids, list(ms)))


class QueryGraph:
    """One query call captured into a CUDA graph (cs_graph_create) over fixed
    device buffers: rewrite `prims` in place, then launch().  Forward graphs
    fill `out` (metric, collide and, per params, count / group outputs);
    adjoint graphs (grad=True) fill `grad_centres`."""

    def __init__(self, scene: Scene, prims, nsigma=1.0, *, prim_type=CS_PRIM_SPHERE,
                 params: QueryParams | None = None, grad=False, grad_out=None, want_count=False):
        torch = _torch()
        params = params or QueryParams()
        self.scene = scene
        self.prims = prims
        assert prims.is_cuda and prims.is_contiguous() and prims.dtype == torch.float32
        cols = 4 if prim_type == CS_PRIM_SPHERE else 10
        Q = prims.numel() // cols
        dev = prims.device
        p = params.to_c()
        self.out = {}
        self.grad_out = grad_out
        if grad:
            self.out["grad_centres"] = torch.empty((Q, 3), dtype=torch.float32, device=dev)
            m = c = None
            g = self.out["grad_centres"]
        else:
            S = len(params.sweep) if len(params.sweep) >= 2 else 1  # n_sigma blocks of a sweep
            m = self.out["metric"] = torch.empty(S * Q, dtype=torch.float32, device=dev)
            c = self.out["collide"] = torch.empty(S * Q, dtype=torch.uint8, device=dev)
            g = None
            if want_count:
                self.out["count"] = torch.empty(S * Q, dtype=torch.int32, device=dev)
                p.out_count = abi.ptr(self.out["count"])
            if params.group_size > 0:
                ng = S * ((Q + params.group_size - 1) // params.group_size)
                self.out["group_metric"] = torch.empty(ng, dtype=torch.float32, device=dev)
                self.out["group_collide"] = torch.empty(ng, dtype=torch.uint8, device=dev)
                p.out_group_metric = abi.ptr(self.out["group_metric"])
                p.out_group_collide = abi.ptr(self.out["group_collide"])
        self._h = ctypes.c_void_p()
        check(abi.cs_graph_create(scene.handle, prim_type, prims, Q, float(nsigma), m, c, grad_out, g, p,
                                  self._h))
        self.kernels = abi.cs_graph_kernels(self._h)

    def launch(self, stream=None):
        check(abi.cs_graph_launch(self._h, stream))
        return self.out

    def sync(self, stream=None):
        check(abi.cs_graph_sync(self._h, stream))

    def close(self):
        if self._h:
            check(abi.cs_graph_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Serving loop over resident scenes (cs_server_*): submit() host numpy
    requests, wait() for their results and timeline."""

    def __init__(self, scenes, *, slots=3, slot_rows=1 << 19, max_requests=4096, tile_config=abi.CS_TILE_TUNED,
                 params: QueryParams | None = None, use_graphs: bool = True):
        params = params or QueryParams()
        self.scenes = list(scenes)
        cfg = abi.cs_server_config()
        check(abi.cs_server_config_init(cfg))
        cfg.slots, cfg.slot_rows, cfg.max_requests, cfg.tile_config = slots, slot_rows, max_requests, tile_config
        cfg.use_graphs = 1 if use_graphs else 0
        cfg.params = params.to_c()
        self._h = ctypes.c_void_p()
        check(abi.cs_server_create([s.handle for s in self.scenes], len(self.scenes), cfg, self._h))
        self._live = {}

    def submit(self, scene: int, prims, nsigma: float, *, prim_type=CS_PRIM_SPHERE, group_size=0,
               want_count=False, out=None) -> int:
        """Queue one request (host float32 [Q,4] or [Q,10]); returns its ticket."""
        import numpy as np
        prims = np.ascontiguousarray(prims, dtype=np.float32)
        cols = 4 if prim_type == CS_PRIM_SPHERE else 10
        Q = prims.size // cols
        if out is None:
            out = {"metric": np.empty(Q, np.float32), "collide": np.empty(Q, np.uint8)}
            if want_count:
                out["count"] = np.empty(Q, np.int32)
            if group_size > 0:
                ng = (Q + group_size - 1) // group_size
                out["group_metric"] = np.empty(ng, np.float32)
                out["group_collide"] = np.empty(ng, np.uint8)
        r = abi.cs_request()
        r.scene, r.prim_type, r.prims, r.Q = scene, prim_type, abi.ptr(prims), Q
        r.conservatism, r.group_size = float(nsigma), int(group_size)
        r.out_metric = abi.ptr(out.get("metric"))
        r.out_collide = abi.ptr(out.get("collide"))
        r.out_count = abi.ptr(out.get("count"))
        r.out_group_metric = abi.ptr(out.get("group_metric"))
        r.out_group_collide = abi.ptr(out.get("group_collide"))
        t = ctypes.c_uint64()
        check(abi.cs_server_submit(self._h, r, t))
        self._live[t.value] = (prims, out)  # the buffers stay alive until wait()
        return t.value

    def wait(self, ticket: int, timeout: float = -1.0):
        """Results (dict of numpy arrays) and timeline of a request."""
        tm = abi.cs_request_times()
        st = abi.cs_server_wait(self._h, ticket, timeout, tm)
        if st == abi.CS_ERR_TIMEOUT and tm.status == 0 and tm.completed == 0:
            raise CsError(st, abi.cs_last_error())
        _, out = self._live.pop(ticket)
        check(st)
        return out, {"submitted": tm.submitted, "launched": tm.launched, "completed": tm.completed,
                     "batch_rows": tm.batch_rows, "batch_requests": tm.batch_requests}

    def stats(self) -> dict:
        s = abi.cs_server_stats()
        check(abi.cs_server_stats_get(self._h, s))
        return {k: getattr(s, k) for k, _ in abi.cs_server_stats._fields_}

    @staticmethod
    def clock() -> float:
        return abi.cs_server_clock()

    def close(self):
        if self._h:
            check(abi.cs_server_destroy(self._h))
            self._h = ctypes.c_void_p()
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _mppi_desc(K, T, dt, radius, nsigma, lam, w_collision, w_goal, w_terminal, w_control, goal):
    d = abi.cs_mppi_desc()
    d.K, d.T, d.dt, d.radius, d.nsigma, d.lambda_ = K, T, dt, radius, nsigma, lam
    d.w_collision, d.w_goal, d.w_terminal, d.w_control = w_collision, w_goal, w_terminal, w_control
    for a in range(3):
        d.goal[a] = goal[a]
    return d


def mppi_step(scene: Scene, x0, U, eps, *, dt=0.1, radius=0.15, nsigma=1.0, lam=1.0, w_collision=10.0,
              w_goal=0.1, w_terminal=1.0, w_control=0.01, goal=(0.0, 0.0, 0.0),
              params: QueryParams | None = None, stream=None, out=None) -> dict:
    """cs_mppi_step on device tensors: x0 [3], U [T,3], eps [K,T,3].
    Returns the updated nominal sequence, per-rollout cost, Eq. 10 weights
    and collision flags (device tensors)."""
    torch = _torch()
    dev = scene.device
    x0 = _as_f32(x0, dev).reshape(3)
    U = _as_f32(U, dev).reshape(-1, 3)
    T = U.shape[0]
    eps = _as_f32(eps, dev).reshape(-1, T, 3)
    K = eps.shape[0]
    if out is None:
        out = {"U": torch.empty((T, 3), dtype=torch.float32, device=dev),
               "cost": torch.empty(K, dtype=torch.float32, device=dev),
               "weights": torch.empty(K, dtype=torch.float32, device=dev),
               "collide": torch.empty(K, dtype=torch.uint8, device=dev)}
    d = _mppi_desc(K, T, dt, radius, nsigma, lam, w_collision, w_goal, w_terminal, w_control, goal)
    p = (params or QueryParams()).to_c()
    p.stream = abi.stream_handle(stream)
    check(abi.cs_mppi_step(scene.handle, d, x0, U, eps, out["U"], out.get("cost"), out.get("weights"),
                           out.get("collide"), p))
    return out


def path_refine(scene: Scene, ctrl, eps, *, M=8, radius=0.05, nsigma=1.0, lam=1.0, w_length=1.0,
                w_collision=10.0, params: QueryParams | None = None, stream=None, out=None) -> dict:
    """cs_path_refine on device tensors: the control points ctrl [N,3] of a
    plan, eps [K,N,3] perturbations (endpoints ignored).  Returns the
    refined control points, per-rollout cost and Eq. 10 weights."""
    torch = _torch()
    dev = scene.device
    ctrl = _as_f32(ctrl, dev).reshape(-1, 3)
    N = ctrl.shape[0]
    eps = _as_f32(eps, dev).reshape(-1, N, 3)
    K = eps.shape[0]
    if out is None:
        out = {"ctrl": torch.empty((N, 3), dtype=torch.float32, device=dev),
               "cost": torch.empty(K, dtype=torch.float32, device=dev),
               "weights": torch.empty(K, dtype=torch.float32, device=dev)}
    d = abi.cs_refine_desc(K, N, M, radius, nsigma, lam, w_length, w_collision)
    p = (params or QueryParams()).to_c()
    p.stream = abi.stream_handle(stream)
    check(abi.cs_path_refine(scene.handle, d, ctrl, eps, out["ctrl"], out.get("cost"), out.get("weights"), p))
    return out


class MppiGraph:
    """One MPPI iteration captured into a CUDA graph (cs_mppi_graph_create)
    over fixed device tensors x0 [3], U [T,3], eps [K,T,3]; each launch()
    reads what they hold then and writes `out` (U_out = U updates in place
    when in_place=True)."""

    def __init__(self, scene: Scene, x0, U, eps, *, in_place=False, dt=0.1, radius=0.15, nsigma=1.0, lam=1.0,
                 w_collision=10.0, w_goal=0.1, w_terminal=1.0, w_control=0.01, goal=(0.0, 0.0, 0.0),
                 params: QueryParams | None = None):
        torch = _torch()
        for t in (x0, U, eps):
            assert t.is_cuda and t.is_contiguous() and t.dtype == torch.float32
        self.x0, self.U, self.eps = x0, U, eps
        T, K = U.shape[0], eps.shape[0]
        dev = U.device
        self.out = {"U": U if in_place else torch.empty((T, 3), dtype=torch.float32, device=dev),
                    "cost": torch.empty(K, dtype=torch.float32, device=dev),
                    "weights": torch.empty(K, dtype=torch.float32, device=dev),
                    "collide": torch.empty(K, dtype=torch.uint8, device=dev)}
        d = _mppi_desc(K, T, dt, radius, nsigma, lam, w_collision, w_goal, w_terminal, w_control, goal)
        p = (params or QueryParams()).to_c()
        self._h = ctypes.c_void_p()
        check(abi.cs_mppi_graph_create(scene.handle, d, x0, U, eps, self.out["U"], self.out["cost"],
                                       self.out["weights"], self.out["collide"], p, self._h))
        self.kernels = abi.cs_graph_kernels(self._h)

    def launch(self, stream=None):
        check(abi.cs_graph_launch(self._h, stream))
        return self.out

    def sync(self, stream=None):
        check(abi.cs_graph_sync(self._h, stream))

    def close(self):
        if self._h:
            check(abi.cs_graph_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class RrtTree:
    """A tree grown by batched RRT extensions (cs_rrt_extend), held in device
    tensors: nodes [capacity,3], parent [capacity] (-1 for the root), count."""

    def __init__(self, scene: Scene, root, *, capacity=1 << 16, step=0.5, radius=0.15, nsigma=1.0, M=16,
                 params: QueryParams | None = None):
        torch = _torch()
        dev = scene.device
        self.scene = scene
        self.nodes = torch.zeros((capacity, 3), dtype=torch.float32, device=dev)
        self.nodes[0] = _as_f32(root, dev).reshape(3)
        self.parent = torch.full((capacity,), -1, dtype=torch.int32, device=dev)
        self.count = torch.ones(1, dtype=torch.int32, device=dev)
        self.capacity, self.step, self.radius, self.nsigma, self.M = capacity, step, radius, nsigma, M
        self.params = params or QueryParams()

    def extend(self, samples, stream=None) -> dict:
        """One extension with B = len(samples); returns the nearest node and
        the free flag of each sample's edge (device tensors)."""
        torch = _torch()
        s = _as_f32(samples, self.scene.device).reshape(-1, 3)
        B = s.shape[0]
        d = abi.cs_rrt_desc()
        d.B, d.M, d.step, d.radius, d.nsigma, d.capacity = B, self.M, self.step, self.radius, self.nsigma, \
            self.capacity
        out = {"nearest": torch.empty(B, dtype=torch.int32, device=s.device),
               "edge_free": torch.empty(B, dtype=torch.uint8, device=s.device)}
        p = self.params.to_c()
        p.stream = abi.stream_handle(stream)
        check(abi.cs_rrt_extend(self.scene.handle, d, self.nodes, self.parent, self.count, s, out["nearest"],
                                out["edge_free"], p))
        out["_samples"] = s
        return out

    def graph(self, B: int) -> "RrtGraph":
        """Capture this tree's extension with B samples (cs_rrt_graph_create)."""
        return RrtGraph(self, B)


class RrtGraph:
    """One extension of an RrtTree captured into a CUDA graph
    (cs_rrt_graph_create): write the next B samples into `samples`, then
    launch(); `nearest` and `edge_free` hold the last launch's results."""

    def __init__(self, tree: RrtTree, B: int):
        torch = _torch()
        dev = tree.scene.device
        self.tree = tree
        self.samples = torch.zeros((B, 3), dtype=torch.float32, device=dev)
        self.nearest = torch.empty(B, dtype=torch.int32, device=dev)
        self.edge_free = torch.empty(B, dtype=torch.uint8, device=dev)
        d = abi.cs_rrt_desc()
        d.B, d.M, d.step, d.radius, d.nsigma, d.capacity = B, tree.M, tree.step, tree.radius, tree.nsigma, \
            tree.capacity
        self._h = ctypes.c_void_p()
        check(abi.cs_rrt_graph_create(tree.scene.handle, d, tree.nodes, tree.parent, tree.count, self.samples,
                                      self.nearest, self.edge_free, tree.params.to_c(), self._h))
        self.kernels = abi.cs_graph_kernels(self._h)

    def launch(self, stream=None):
        check(abi.cs_graph_launch(self._h, stream))

    def sync(self, stream=None):
        check(abi.cs_graph_sync(self._h, stream))

    def close(self):
        if self._h:
            check(abi.cs_graph_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


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
