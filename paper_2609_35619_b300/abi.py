"""ctypes binding of libcs_b300.so: one Python function per C entry point
(same names, same argument order), argument marshalling only.

Arrays may be torch tensors (device pointers: CUDA tensors; host pointers:
CPU tensors, pinned for asynchronous copies) or numpy arrays (host).  Every
call returns the cs_status code; use `check(status)` to raise on failure.
The library must have been built (``python -m paper_2609_35619_b300.build``);
importing this module on a machine without it raises immediately.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# CS_B300_LIBRARY may name the bounds-checked build of the same sources
# (libcs_b300_debug.so, `python -m paper_2609_35619_b300.build --debug`)
LIB_PATH = os.environ.get("CS_B300_LIBRARY") or os.path.join(HERE, "libcs_b300.so")
DEBUG_LIB_PATH = os.path.join(HERE, "libcs_b300_debug.so")

CS_OK, CS_ERR_INVALID_ARG, CS_ERR_NO_MEMORY, CS_ERR_CUDA, CS_ERR_TIMEOUT, CS_ERR_BAD_HANDLE, \
    CS_ERR_UNSUPPORTED, CS_ERR_BOUNDS = 0, -1, -2, -3, -4, -5, -6, -7
CS_PRIM_SPHERE, CS_PRIM_ELLIPSOID = 0, 1
CS_METRIC_MEAN_COST, CS_METRIC_SUM_COST, CS_METRIC_MIN_S2, CS_METRIC_SOFTMIN_S2, CS_METRIC_FLAGS = 0, 1, 2, 3, 4

STATUS_NAMES = {0: "CS_OK", -1: "CS_ERR_INVALID_ARG", -2: "CS_ERR_NO_MEMORY", -3: "CS_ERR_CUDA",
                -4: "CS_ERR_TIMEOUT", -5: "CS_ERR_BAD_HANDLE", -6: "CS_ERR_UNSUPPORTED", -7: "CS_ERR_BOUNDS"}


class cs_scene_desc(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("means", ctypes.c_void_p),
        ("scales", ctypes.c_void_p),
        ("quats", ctypes.c_void_p),
        ("opacity", ctypes.c_void_p),
        ("on_device", ctypes.c_int32),
        ("use_filter", ctypes.c_int32),
        ("opacity_min", ctypes.c_float),
        ("extent_max", ctypes.c_float),
        ("cell_size", ctypes.c_float),
        ("tier_quantile", ctypes.c_float),
    ]


class cs_params(ctypes.Structure):
    _fields_ = [
        ("gamma", ctypes.c_float),
        ("d_max", ctypes.c_float),
        ("s_min", ctypes.c_float),
        ("eps", ctypes.c_float),
        ("tau", ctypes.c_float),
        ("k_thr", ctypes.c_int32),
        ("mode", ctypes.c_int32),
        ("group_size", ctypes.c_int32),
        ("host_io", ctypes.c_int32),
        ("tile_config", ctypes.c_int32),
        ("nsigma_per_query", ctypes.c_void_p),
        ("stream", ctypes.c_void_p),
        ("out_count", ctypes.c_void_p),
        ("out_group_metric", ctypes.c_void_p),
        ("out_group_collide", ctypes.c_void_p),
        ("out_pair_stats", ctypes.c_void_p),
        ("eval_events", ctypes.c_void_p * 2),
        ("out_kernel_stats", ctypes.c_void_p),
        ("exact_variance", ctypes.c_int32),
        ("sweep_count", ctypes.c_int32),
        ("sweep_nsigma", ctypes.c_float * 8),
    ]


class cs_scene_info(ctypes.Structure):
    _fields_ = [
        ("n_input", ctypes.c_int64),
        ("n_kept", ctypes.c_int64),
        ("n_grid", ctypes.c_int64),
        ("n_large", ctypes.c_int64),
        ("n_invalid", ctypes.c_int64),
        ("dims", ctypes.c_int32 * 3),
        ("cell_size", ctypes.c_float),
        ("sigma_tier", ctypes.c_float),
        ("lo", ctypes.c_float * 3),
        ("hi", ctypes.c_float * 3),
        ("device_bytes", ctypes.c_int64),
    ]


class cs_server_config(ctypes.Structure):
    _fields_ = [
        ("slots", ctypes.c_int32),
        ("slot_rows", ctypes.c_int64),
        ("max_requests", ctypes.c_int32),
        ("tile_config", ctypes.c_int32),
        ("params", cs_params),
        ("use_graphs", ctypes.c_int32),
    ]


class cs_request(ctypes.Structure):
    _fields_ = [
        ("scene", ctypes.c_int32),
        ("prim_type", ctypes.c_int32),
        ("prims", ctypes.c_void_p),
        ("Q", ctypes.c_int64),
        ("conservatism", ctypes.c_float),
        ("group_size", ctypes.c_int32),
        ("out_metric", ctypes.c_void_p),
        ("out_collide", ctypes.c_void_p),
        ("out_count", ctypes.c_void_p),
        ("out_group_metric", ctypes.c_void_p),
        ("out_group_collide", ctypes.c_void_p),
    ]


class cs_request_times(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_double),
        ("launched", ctypes.c_double),
        ("completed", ctypes.c_double),
        ("batch_rows", ctypes.c_int64),
        ("batch_requests", ctypes.c_int64),
        ("status", ctypes.c_int32),
    ]


class cs_server_stats(ctypes.Structure):
    _fields_ = [
        ("batches", ctypes.c_int64),
        ("rows", ctypes.c_int64),
        ("requests", ctypes.c_int64),
        ("max_batch_rows", ctypes.c_int64),
        ("max_batch_requests", ctypes.c_int64),
        ("pending", ctypes.c_int64),
        ("busy_slots", ctypes.c_int64),
    ]


class cs_mppi_desc(ctypes.Structure):
    _fields_ = [
        ("K", ctypes.c_int32),
        ("T", ctypes.c_int32),
        ("dt", ctypes.c_float),
        ("radius", ctypes.c_float),
        ("nsigma", ctypes.c_float),
        ("lambda_", ctypes.c_float),
        ("w_collision", ctypes.c_float),
        ("w_goal", ctypes.c_float),
        ("w_terminal", ctypes.c_float),
        ("w_control", ctypes.c_float),
        ("goal", ctypes.c_float * 3),
    ]


class cs_rrt_desc(ctypes.Structure):
    _fields_ = [
        ("B", ctypes.c_int32),
        ("M", ctypes.c_int32),
        ("step", ctypes.c_float),
        ("radius", ctypes.c_float),
        ("nsigma", ctypes.c_float),
        ("capacity", ctypes.c_int32),
    ]


class cs_refine_desc(ctypes.Structure):
    _fields_ = [
        ("K", ctypes.c_int32),
        ("N", ctypes.c_int32),
        ("M", ctypes.c_int32),
        ("radius", ctypes.c_float),
        ("nsigma", ctypes.c_float),
        ("lam", ctypes.c_float),
        ("w_length", ctypes.c_float),
        ("w_collision", ctypes.c_float),
    ]


class cs_render_desc(ctypes.Structure):
    _fields_ = [
        ("n_views", ctypes.c_int32),
        ("width", ctypes.c_int32),
        ("height", ctypes.c_int32),
        ("near_plane", ctypes.c_float),
        ("dilation", ctypes.c_float),
        ("background", ctypes.c_float * 3),
        ("stream", ctypes.c_void_p),
        ("out_instances", ctypes.POINTER(ctypes.c_int64)),
    ]


CS_TILE_TUNED = -1

_P = ctypes.c_void_p
_SIGNATURES = {
    "cs_params_init": (ctypes.c_int, [ctypes.POINTER(cs_params)]),
    "cs_scene_create": (ctypes.c_int, [ctypes.POINTER(cs_scene_desc), _P, ctypes.POINTER(_P)]),
    "cs_scene_destroy": (ctypes.c_int, [_P]),
    "cs_scene_info_get": (ctypes.c_int, [_P, ctypes.POINTER(cs_scene_info)]),
    "cs_scene_export": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "cs_scene_save": (ctypes.c_int, [_P, ctypes.c_char_p, _P]),
    "cs_scene_load": (ctypes.c_int, [ctypes.c_char_p, _P, ctypes.POINTER(_P)]),
    "cs_query": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int64, ctypes.c_float, _P, _P,
                                ctypes.POINTER(cs_params)]),
    "cs_query_grad": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int64, ctypes.c_float, _P, _P,
                                     ctypes.POINTER(cs_params)]),
    "cs_query_noalloc": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int64, ctypes.c_float, _P, _P,
                                        ctypes.POINTER(cs_params)]),
    "cs_query_fwd_grad": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int64, ctypes.c_float, _P, _P, _P, _P,
                                         ctypes.POINTER(cs_params)]),
    "cs_pose_spheres": (ctypes.c_int, [_P, ctypes.c_int64, _P, ctypes.c_int32, ctypes.c_float, _P, _P]),
    "cs_pose_spheres_grad": (ctypes.c_int, [_P, ctypes.c_int64, _P, ctypes.c_int32, _P, _P, _P]),
    "cs_sync": (ctypes.c_int, [_P, _P]),
    "cs_graph_create": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int64, ctypes.c_float, _P, _P, _P, _P,
                                       ctypes.POINTER(cs_params), ctypes.POINTER(_P)]),
    "cs_mppi_graph_create": (ctypes.c_int, [_P, ctypes.POINTER(cs_mppi_desc), _P, _P, _P, _P, _P, _P, _P,
                                            ctypes.POINTER(cs_params), ctypes.POINTER(_P)]),
    "cs_rrt_graph_create": (ctypes.c_int, [_P, ctypes.POINTER(cs_rrt_desc), _P, _P, _P, _P, _P, _P,
                                           ctypes.POINTER(cs_params), ctypes.POINTER(_P)]),
    "cs_graph_launch": (ctypes.c_int, [_P, _P]),
    "cs_graph_sync": (ctypes.c_int, [_P, _P]),
    "cs_graph_kernels": (ctypes.c_int64, [_P]),
    "cs_graph_destroy": (ctypes.c_int, [_P]),
    "cs_autotune": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int64, ctypes.c_float,
                                   ctypes.POINTER(cs_params), ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                   _P, ctypes.c_int32]),
    "cs_autotune_log": (ctypes.c_int, [ctypes.c_char_p]),
    "cs_mppi_step": (ctypes.c_int, [_P, ctypes.POINTER(cs_mppi_desc), _P, _P, _P, _P, _P, _P, _P,
                                    ctypes.POINTER(cs_params)]),
    "cs_rrt_extend": (ctypes.c_int, [_P, ctypes.POINTER(cs_rrt_desc), _P, _P, _P, _P, _P, _P,
                                     ctypes.POINTER(cs_params)]),
    "cs_path_refine": (ctypes.c_int, [_P, ctypes.POINTER(cs_refine_desc), _P, _P, _P, _P, _P,
                                      ctypes.POINTER(cs_params)]),
    "cs_render_desc_init": (ctypes.c_int, [ctypes.POINTER(cs_render_desc)]),
    "cs_scene_set_appearance": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32, _P]),
    "cs_render": (ctypes.c_int, [_P, ctypes.POINTER(cs_render_desc), _P, _P, _P, _P]),
    "cs_server_config_init": (ctypes.c_int, [ctypes.POINTER(cs_server_config)]),
    "cs_server_create": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(cs_server_config), ctypes.POINTER(_P)]),
    "cs_server_submit": (ctypes.c_int, [_P, ctypes.POINTER(cs_request), ctypes.POINTER(ctypes.c_uint64)]),
    "cs_server_wait": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(cs_request_times)]),
    "cs_server_stats_get": (ctypes.c_int, [_P, ctypes.POINTER(cs_server_stats)]),
    "cs_server_clock": (ctypes.c_double, []),
    "cs_server_destroy": (ctypes.c_int, [_P]),
    "cs_tile_configs": (ctypes.c_int32, [_P, ctypes.c_int32]),
    "cs_selftest_wait_timeout": (ctypes.c_int, [ctypes.c_int64, _P]),
    "cs_launch_count": (ctypes.c_int64, []),
    "cs_release_scratch": (ctypes.c_int, []),
    "cs_last_error": (ctypes.c_char_p, []),
    "cs_version": (ctypes.c_char_p, []),
}

_lib = None


def load():
    """Load libcs_b300.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2609_35619_b300.build` (there is no fallback path)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def symbols():
    return list(_SIGNATURES)


class CsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status: int) -> int:
    if status != CS_OK:
        raise CsError(status, cs_last_error())
    return status


def ptr(x) -> int | None:
    """Address of a tensor/array (None -> NULL).  Must be contiguous."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):  # torch.Tensor
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr() if x.numel() > 0 else None
    if hasattr(x, "ctypes"):  # numpy
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data if x.size > 0 else None
    raise TypeError(f"cannot take the address of {type(x)}")


def stream_handle(stream) -> int | None:
    """cudaStream_t of a torch stream (None -> the current torch stream)."""
    if stream is None:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream or None
        return None
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None


# ------------------------------------------------ one function per entry point
def cs_params_init(p: cs_params) -> int:
    return load().cs_params_init(ctypes.byref(p))


def cs_scene_create(desc: cs_scene_desc, stream, out: ctypes.c_void_p) -> int:
    return load().cs_scene_create(ctypes.byref(desc), stream_handle(stream), ctypes.byref(out))


def cs_scene_destroy(scene) -> int:
    return load().cs_scene_destroy(scene)


def cs_scene_info_get(scene, info: cs_scene_info) -> int:
    return load().cs_scene_info_get(scene, ctypes.byref(info))


def cs_scene_export(scene, pos, cov, index, stream) -> int:
    return load().cs_scene_export(scene, ptr(pos), ptr(cov), ptr(index), stream_handle(stream))


def cs_scene_save(scene, path, stream) -> int:
    return load().cs_scene_save(scene, None if path is None else os.fsencode(path), stream_handle(stream))


def cs_scene_load(path, stream, out: "ctypes.c_void_p") -> int:
    return load().cs_scene_load(None if path is None else os.fsencode(path), stream_handle(stream),
                                ctypes.byref(out))


def cs_query(scene, prim_type, prims, Q, conservatism, out_metric, out_collide, params) -> int:
    return load().cs_query(scene, prim_type, ptr(prims), int(Q), float(conservatism), ptr(out_metric),
                           ptr(out_collide), None if params is None else ctypes.byref(params))


def cs_query_noalloc(scene, prim_type, prims, Q, conservatism, out_metric, out_collide, params) -> int:
    return load().cs_query_noalloc(scene, prim_type, ptr(prims), int(Q), float(conservatism),
                                   ptr(out_metric), ptr(out_collide),
                                   None if params is None else ctypes.byref(params))


CS_QUERY_NOALLOC_MAX_ROWS = 65536


def cs_query_grad(scene, prim_type, prims, Q, conservatism, grad_out, grad_centres, params) -> int:
    return load().cs_query_grad(scene, prim_type, ptr(prims), int(Q), float(conservatism),
                                ptr(grad_out), ptr(grad_centres),
                                None if params is None else ctypes.byref(params))


def cs_query_fwd_grad(scene, prim_type, prims, Q, conservatism, grad_out, out_metric, out_collide, grad_centres,
                      params) -> int:
    return load().cs_query_fwd_grad(scene, prim_type, ptr(prims), int(Q), float(conservatism), ptr(grad_out),
                                    ptr(out_metric), ptr(out_collide), ptr(grad_centres),
                                    None if params is None else ctypes.byref(params))


def cs_pose_spheres(poses, P, offsets, K, radius, out_spheres, stream) -> int:
    return load().cs_pose_spheres(ptr(poses), int(P), ptr(offsets), int(K), float(radius),
                                  ptr(out_spheres), stream_handle(stream))


def cs_pose_spheres_grad(poses, P, offsets, K, grad_centres, grad_poses, stream) -> int:
    return load().cs_pose_spheres_grad(ptr(poses), int(P), ptr(offsets), int(K), ptr(grad_centres),
                                       ptr(grad_poses), stream_handle(stream))


def cs_sync(scene, stream) -> int:
    return load().cs_sync(scene, stream_handle(stream))


def cs_graph_create(scene, prim_type, prims, Q, conservatism, out_metric, out_collide, grad_out,
                    grad_centres, params, out: ctypes.c_void_p) -> int:
    return load().cs_graph_create(scene, prim_type, ptr(prims), int(Q), float(conservatism), ptr(out_metric),
                                  ptr(out_collide), ptr(grad_out), ptr(grad_centres),
                                  None if params is None else ctypes.byref(params), ctypes.byref(out))


def cs_rrt_graph_create(scene, desc, nodes, parent, count, samples, nearest, edge_free, params,
                        out: ctypes.c_void_p) -> int:
    return load().cs_rrt_graph_create(scene, ctypes.byref(desc), ptr(nodes), ptr(parent), ptr(count), ptr(samples),
                                      ptr(nearest), ptr(edge_free), None if params is None else ctypes.byref(params),
                                      ctypes.byref(out))


def cs_mppi_graph_create(scene, desc, x0, U, eps, U_out, cost, weights, collide, params,
                         out: ctypes.c_void_p) -> int:
    return load().cs_mppi_graph_create(scene, ctypes.byref(desc), ptr(x0), ptr(U), ptr(eps), ptr(U_out), ptr(cost),
                                       ptr(weights), ptr(collide), None if params is None else ctypes.byref(params),
                                       ctypes.byref(out))


def cs_graph_launch(graph, stream) -> int:
    return load().cs_graph_launch(graph, stream_handle(stream))


def cs_graph_sync(graph, stream) -> int:
    return load().cs_graph_sync(graph, stream_handle(stream))


def cs_graph_kernels(graph) -> int:
    return int(load().cs_graph_kernels(graph))


def cs_graph_destroy(graph) -> int:
    return load().cs_graph_destroy(graph)


def cs_autotune(scene, prim_type, prims, Q, conservatism, params, reps, best: ctypes.c_int32, ms, cap) -> int:
    return load().cs_autotune(scene, prim_type, ptr(prims), int(Q), float(conservatism),
                              None if params is None else ctypes.byref(params), int(reps), ctypes.byref(best),
                              ptr(ms), int(cap))


def cs_autotune_log(path) -> int:
    return load().cs_autotune_log(None if path is None else os.fsencode(path))


def cs_mppi_step(scene, desc: cs_mppi_desc, x0, U, eps, U_out, cost, weights, collide, params) -> int:
    return load().cs_mppi_step(scene, ctypes.byref(desc), ptr(x0), ptr(U), ptr(eps), ptr(U_out), ptr(cost),
                               ptr(weights), ptr(collide), None if params is None else ctypes.byref(params))


def cs_rrt_extend(scene, desc: cs_rrt_desc, nodes, parent, count, samples, nearest, edge_free, params) -> int:
    return load().cs_rrt_extend(scene, ctypes.byref(desc), ptr(nodes), ptr(parent), ptr(count), ptr(samples),
                                ptr(nearest), ptr(edge_free), None if params is None else ctypes.byref(params))


def cs_path_refine(scene, desc: cs_refine_desc, ctrl, eps, ctrl_out, cost, weights, params) -> int:
    return load().cs_path_refine(scene, ctypes.byref(desc), ptr(ctrl), ptr(eps), ptr(ctrl_out), ptr(cost),
                                 ptr(weights), None if params is None else ctypes.byref(params))


def cs_render_desc_init(desc: cs_render_desc) -> int:
    return load().cs_render_desc_init(ctypes.byref(desc))


def cs_scene_set_appearance(scene, opacity, colors, on_device, stream) -> int:
    return load().cs_scene_set_appearance(scene, ptr(opacity), ptr(colors), int(on_device), stream_handle(stream))


def cs_render(scene, desc: cs_render_desc, cams, rgb, depth, alpha) -> int:
    return load().cs_render(scene, ctypes.byref(desc), ptr(cams), ptr(rgb), ptr(depth), ptr(alpha))


def cs_server_config_init(cfg: cs_server_config) -> int:
    return load().cs_server_config_init(ctypes.byref(cfg))


def cs_server_create(scenes, n_scenes, cfg, out: ctypes.c_void_p) -> int:
    arr = (ctypes.c_void_p * max(1, int(n_scenes)))(*[s if isinstance(s, int) else s.value for s in scenes])
    return load().cs_server_create(ctypes.cast(arr, ctypes.c_void_p), int(n_scenes),
                                   None if cfg is None else ctypes.byref(cfg), ctypes.byref(out))


def cs_server_submit(server, req: cs_request, ticket: ctypes.c_uint64) -> int:
    return load().cs_server_submit(server, ctypes.byref(req), ctypes.byref(ticket))


def cs_server_wait(server, ticket, timeout_s, times) -> int:
    return load().cs_server_wait(server, int(ticket), float(timeout_s),
                                 None if times is None else ctypes.byref(times))


def cs_server_stats_get(server, out: cs_server_stats) -> int:
    return load().cs_server_stats_get(server, ctypes.byref(out))


def cs_server_clock() -> float:
    return float(load().cs_server_clock())


def cs_server_destroy(server) -> int:
    return load().cs_server_destroy(server)


def cs_tile_configs() -> list:
    lib = load()
    n = lib.cs_tile_configs(None, 0)
    buf = (ctypes.c_int32 * max(n, 1))()
    lib.cs_tile_configs(ctypes.cast(buf, ctypes.c_void_p), n)
    return list(buf[:n])


def cs_selftest_wait_timeout(spins: int, stream) -> int:
    return load().cs_selftest_wait_timeout(int(spins), stream_handle(stream))


def cs_release_scratch() -> int:
    return load().cs_release_scratch()


def cs_launch_count() -> int:
    return int(load().cs_launch_count())


def cs_last_error() -> str:
    return load().cs_last_error().decode()


def cs_version() -> str:
    return load().cs_version().decode()
