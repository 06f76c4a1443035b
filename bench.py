#!/usr/bin/env python
"""Benchmark of the collision-metric hot path on B300; prints ONE JSON line.

Workload (one step = every stage of the hot path over one batch):
  the 1M-Gaussian tabletop scene (plane + 25 object clusters) built from
  device-resident arrays (Eq. 2 repack, floater filter, grid, large tier);
  262,144 arm spheres (4,096 configurations x 64, per-configuration sums) and
  2,097,152 RRT edge spheres (2,048 edges x 16 strides x 64, per-edge OR),
  each at n_sigma in {0, 0.5, 1, 2}; then 512 trajectories x 64 waypoint
  poses x 8 body spheres: pose chain, metric, adjoint and pose adjoint.
Metric: useful (query, Gaussian) pair evaluations per second (pairs inside the
neighbour sets), with queries/s beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs the same workload on its own GPU
(independent replicas, weak scaling); the job value is the pairs of all ranks
over the slowest rank's time.  --impl reference times the FP64 CPU oracle on
the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NSIGMAS = (0.0, 0.5, 1.0, 2.0)
# the counters of cs_params.out_kernel_stats, in order
KSTAT_NAMES = ["stages", "chunks_tested", "chunks_pass_warp", "hits", "chunks_staged", "stages_filled",
               "consumer_polls", "producer_polls", "consumer_cycles", "consumer_wait_cycles",
               "producer_cycles", "producer_wait_cycles", "consumer_first_cycles", "producer_first_cycles",
               "consumer_tail_cycles", "tiles"]
OPS_PER_PAIR = 26  # canonical FP32 ops of one sphere pair (see the design notes)
# DRAM bytes (read + write) per forward launch of the fused kernel: the mean of
# the step's two sweep launches from the ncu captures summarised under
# profiles/ (arm 41.21 MB, edge 124.02 MB), valid for the library version they
# were taken with (reported as null otherwise)
TRAFFIC = {"version": "cs_b300 1.5 (sm_103a)", "bytes": (41.13024e6 + 0.076544e6 + 97.350912e6 + 26.670592e6) / 2,
           "case": "mean of the step's two forward sweep launches, tile 30 (arm 262,144 x 4 rows: 41.2 MB; "
                   "edge 2,097,152 x 4 rows: 124.0 MB)"}
WORKLOAD = ("tabletop-1M: 262,144 arm + 2,097,152 edge spheres x n_sigma{0,0.5,1,2} + 262,144 pose spheres "
            "fwd+adjoint (each batch's conservatism sweep as one launch; the pose forward and adjoint as one fused launch)")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tiles", default="",
                    help="ARM,EDGE tile ids for the step (default: chosen by the autotuner before timing)")
    ap.add_argument("--serve-requests", type=int, default=1500,
                    help="requests per load (25, 50, 75 and 90 %% of the served capacity) of the serving "
                         "measurement in the default run")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-requests-sweep", type=int, default=10_000, help="requests per load in --case serve")
    ap.add_argument("--serve-eager", action="store_true",
                    help="--case serve: launch the query path's kernels one by one instead of replaying graphs")
    ap.add_argument("--serve-slots", type=int, default=3, help="server batch slots in --case serve")
    ap.add_argument("--serve-rows", type=int, default=1 << 19, help="rows per server slot in --case serve")
    ap.add_argument("--no-per-call", action="store_true", help="--case serve: skip the per-call baseline")
    ap.add_argument("--case", default="step",
                    choices=["step", "eval", "serve", "mppi", "rrt", "variants", "render", "build"],
                    help="eval: the profiling case -- build the tabletop scene, then one warm-up "
                         "and one measured query of the 262,144 arm spheres at n_sigma=1 "
                         "(two fused-kernel launches); prints a short JSON summary. "
                         "serve: the serving sweep (two 3M apartment scenes, Poisson arrivals at "
                         "25/50/75/90 %% of the served capacity, 10,000 requests per load)")
    ap.add_argument("--tile", type=int, default=0, help="tile configuration for --case eval (0 = auto)")
    ap.add_argument("--batch", default="arm", choices=["arm", "edge", "arm_ellipsoids"],
                    help="query batch for --case eval (arm_ellipsoids: 229,376 link ellipsoids, groups of 7)")
    ap.add_argument("--nsigma", type=float, default=1.0, help="n_sigma for --case eval")
    ap.add_argument("--grad", action="store_true", help="--case eval: time the adjoint kernel instead")
    ap.add_argument("--fused", action="store_true",
                    help="--case eval with --grad: the fused forward and adjoint (cs_query_fwd_grad)")
    ap.add_argument("--flags", action="store_true", help="--case eval: collision flags only (early exit)")
    ap.add_argument("--sweep", action="store_true",
                    help="--case eval: the four n_sigma values of the step in one launch (rows repeated, n_sigma "
                         "per row) against four separate launches")
    ap.add_argument("--cell", type=float, default=0.0,
                    help="--case eval: chunk extent limit of the scene build (0 = automatic)")
    ap.add_argument("--exact", action="store_true",
                    help="--case eval: exact variance of the quadratic form in Eq. 8 (cs_params.exact_variance)")
    return ap.parse_args()


def make_inputs():
    import cs_synth as S
    scene = S.tabletop_scene()
    arm = S.arm_queries()
    edge = S.edge_queries()
    poses, offs, radius = S.trajectory_poses()
    return scene, arm, edge, poses, offs, radius


# --------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ ours
def run_ours(args, rank, world):
    import torch

    import paper_2609_35619_b300 as cs

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    scene_h, arm_h, edge_h, poses_h, offs_h, radius = make_inputs()
    torch.cuda.synchronize(dev)
    free_start, _ = torch.cuda.mem_get_info(dev)  # before any of the job's device memory
    with torch.cuda.stream(stream):
        d_scene = {k: torch.as_tensor(v, device=dev) for k, v in scene_h.items()}
        d_arm = torch.as_tensor(arm_h, device=dev)
        d_edge = torch.as_tensor(edge_h, device=dev)
        d_poses = torch.as_tensor(poses_h, device=dev)
        d_offs = torch.as_tensor(offs_h, device=dev)
        K = offs_h.shape[0]
        n_pose = poses_h.shape[0]
        ones = torch.ones(n_pose, dtype=torch.float32, device=dev)
        outs = {}
        for name, q, G in (("arm", d_arm, 64), ("edge", d_edge, 1024)):
            Q = len(NSIGMAS) * q.shape[0]  # one block of outputs per n_sigma of the sweep
            outs[name] = {"metric": torch.empty(Q, device=dev), "collide": torch.empty(Q, dtype=torch.uint8, device=dev),
                          "group_metric": torch.empty((Q + G - 1) // G, device=dev),
                          "group_collide": torch.empty((Q + G - 1) // G, dtype=torch.uint8, device=dev)}
        pose_out = {"metric": torch.empty(n_pose * K, device=dev),
                    "collide": torch.empty(n_pose * K, dtype=torch.uint8, device=dev),
                    "group_metric": torch.empty(n_pose, device=dev),
                    "group_collide": torch.empty(n_pose, dtype=torch.uint8, device=dev),
                    "grad": torch.empty((n_pose * K, 3), device=dev)}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    torch.cuda.synchronize(dev)

    # tile shapes for the two batch classes from the autotuner (untimed)
    if args.tiles:
        tt = [int(x) for x in args.tiles.split(",")]
        tiles = {"arm": tt[0], "edge": tt[1], "source": "--tiles"}
    else:
        tune_scene = cs.Scene(d_scene["means"], d_scene["scales"], d_scene["quats"], d_scene["opacity"],
                              device=dev, stream=stream)
        sw = cs.QueryParams(sweep=NSIGMAS)
        tiles = {"arm": tune_scene.autotune(d_arm, 0.0, params=sw, reps=2, stream=stream)[0],
                 "edge": tune_scene.autotune(d_edge, 0.0, params=sw, reps=1, stream=stream)[0],
                 "source": "cs_autotune"}
        tune_scene.close()

    def step(events=None, stats=None, build_ev=None):
        ev = iter(events) if events is not None else None
        nxt = (lambda: (next(ev), next(ev))) if ev is not None else (lambda: None)
        if build_ev is not None:
            build_ev[0].record(stream)
        scene = cs.Scene(d_scene["means"], d_scene["scales"], d_scene["quats"], d_scene["opacity"],
                         device=dev, stream=stream)
        if build_ev is not None:
            build_ev[1].record(stream)
        # the conservatism sweep: one launch per batch for all four n_sigma values
        scene.query(d_arm, 0.0, params=cs.QueryParams(group_size=64, tile_config=tiles["arm"], sweep=NSIGMAS),
                    stream=stream, eval_events=nxt(), out=outs["arm"], pair_stats=stats)
        scene.query(d_edge, 0.0, params=cs.QueryParams(group_size=1024, tile_config=tiles["edge"], sweep=NSIGMAS),
                    stream=stream, eval_events=nxt(), out=outs["edge"], pair_stats=stats)
        with torch.cuda.stream(stream):
            sph = cs.pose_spheres(d_poses, d_offs, radius, stream=stream)
            # forward (metric, flag, per-pose cost) and adjoint in one fused launch
            scene.query_fwd_grad(sph, 1.0, grad_out=ones, params=cs.QueryParams(group_size=K), stream=stream,
                                 eval_events=nxt(), out=pose_out, pair_stats=stats)
            gp = cs.pose_spheres_grad(d_poses, d_offs, pose_out["grad"], stream=stream)
        return scene, gp

    # ---- pair counts of one step (untimed, with the stats counters on)
    stats = torch.zeros(2, dtype=torch.int64, device=dev)
    sc, _ = step(stats=stats)
    torch.cuda.synchronize(dev)
    cand_pairs, useful_pairs = (int(x) for x in stats.cpu().tolist())
    # forward sphere launches only (the roofline's kernel): rerun without the grad pass
    stats_fwd = torch.zeros(2, dtype=torch.int64, device=dev)
    sc.query(d_arm, 0.0, params=cs.QueryParams(group_size=64, tile_config=tiles["arm"], sweep=NSIGMAS),
             stream=stream, out=outs["arm"], pair_stats=stats_fwd)
    sc.query(d_edge, 0.0, params=cs.QueryParams(group_size=1024, tile_config=tiles["edge"], sweep=NSIGMAS),
             stream=stream, out=outs["edge"], pair_stats=stats_fwd)
    torch.cuda.synchronize(dev)
    fwd_cand, fwd_useful = (int(x) for x in stats_fwd.cpu().tolist())
    info = sc.info()
    sc.close()
    n_queries = len(NSIGMAS) * (arm_h.shape[0] + edge_h.shape[0]) + 2 * n_pose * K
    n_fwd_launches = 2

    for _ in range(args.warmup):
        s, _ = step()
        torch.cuda.synchronize(dev)
        s.close()

    dist = world > 1
    if dist:
        import torch.distributed as tdist
    clocks = ClockSampler(dev.index)
    clocks.start()
    total_ms = 0.0
    build_ms = []
    eval_ms = []  # per forward-sphere launch of the tabletop sweep
    l0 = cs.abi.cs_launch_count()
    free_min = torch.cuda.mem_get_info(dev)[0]
    scene_bytes = 0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize(dev)
        if dist:
            tdist.barrier()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(2 * (n_fwd_launches + 2))]
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        bev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        t0.record(stream)
        s, _ = step(events=evs, build_ev=bev)
        t1.record(stream)
        torch.cuda.synchronize(dev)
        scene_bytes = s.info()["device_bytes"]
        free_min = min(free_min, torch.cuda.mem_get_info(dev)[0])
        s.close()
        total_ms += t0.elapsed_time(t1)
        build_ms.append(bev[0].elapsed_time(bev[1]))
        for k in range(n_fwd_launches):
            eval_ms.append(evs[2 * k].elapsed_time(evs[2 * k + 1]))
    launches = cs.abi.cs_launch_count() - l0
    clk = clocks.stop()
    ms_step = total_ms / args.steps
    if dist:
        t = torch.tensor([ms_step], device=dev)
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        ms_step = float(t.item())
    value = world * useful_pairs / (ms_step * 1e-3)
    qps = world * n_queries / (ms_step * 1e-3)

    # ---- roofline of the fused forward kernel (FP32 pipe bound)
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    max_mhz = float(peaks.get("sm_max_mhz", 2032.0))
    peak_ops = sms * 128 * max_mhz * 1e6  # FP32 lanes x max SM clock
    avg_eval_s = (sum(eval_ms) / len(eval_ms)) * 1e-3
    ops_per_launch = fwd_useful / n_fwd_launches * OPS_PER_PAIR
    achieved = ops_per_launch / avg_eval_s
    roofline = {"bound": "alu", "kernel": "k_eval<sphere> (fused cull+evaluate+reduce)",
                "achieved": achieved / 1e12, "peak": peak_ops / 1e12, "unit": "TFLOP/s",
                "frac": achieved / peak_ops,
                "traffic": TRAFFIC["bytes"] if cs.abi.cs_version() == TRAFFIC["version"] else None,
                "traffic_case": TRAFFIC["case"],
                "peak_basis": f"{sms} SMs x 128 FP32 lanes x {max_mhz:.0f} MHz (max SM clock)",
                "ops_per_pair": OPS_PER_PAIR, "useful_pairs_per_launch": fwd_useful / n_fwd_launches,
                "candidate_pairs_per_launch": fwd_cand / n_fwd_launches,
                "avg_launch_ms": avg_eval_s * 1e3,
                "candidate_frac": (fwd_cand * OPS_PER_PAIR / n_fwd_launches / avg_eval_s) / peak_ops}

    # scene build (Eq. 2 repack, filter, Hilbert order, chunks, tree): minimal
    # traffic is the 44 input bytes read and the 40-byte record written per
    # Gaussian; the build synchronises the host a few times, so this is a
    # lower bound of the build's own bandwidth
    n_g = int(scene_h["means"].shape[0])
    b_ms = sum(build_ms) / len(build_ms)
    build = {"ms": b_ms, "algorithmic_bytes": n_g * 84, "achieved_gbs": n_g * 84 / (b_ms * 1e-3) / 1e9,
             "peak_gbs": float(peaks.get("hbm_gbs", 6400.0)),
             "note": "44 B read + 40 B written per Gaussian over the whole build (host syncs included)"}
    build["frac"] = build["achieved_gbs"] / build["peak_gbs"]

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, cs, torch, dev, stream, scene_h, arm_h, edge_h, poses_h, offs_h, radius,
                      useful_pairs, world, tiles)

    result = {
        "metric": "query-Gaussian pair evals/s (useful pairs inside the neighbour sets)",
        "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_gaussians": int(scene_h["means"].shape[0]),
                   "n_kept": info["n_kept"], "queries_per_step": n_queries,
                   "useful_pairs_per_step": useful_pairs, "candidate_pairs_per_step": cand_pairs,
                   "nsigma": list(NSIGMAS), "parallelism": f"replicas x{world}",
                   "l2": "256 MB buffer written between steps (outside the timed region)",
                   "grid": {"dims": info["dims"], "cell_size": info["cell_size"],
                            "n_large": info["n_large"]}},
        "queries_per_s": qps, "roofline": roofline, "build": build, "tiles": tiles, "e2e": e2e, "clocks": clk,
        "vram": {"scene_bytes": int(scene_bytes), "job_device_bytes": int(free_start - free_min),
                 "note": "scene = the resident 1M-Gaussian scene (chunk blocks, tree, export arrays); job = device "
                         "memory in use at the end of a timed step minus that before the job's first allocation "
                         "(inputs, outputs, 256 MB L2 flush buffer, scene, the library's query scratch)"},
        "gpu_launches": int(launches // args.steps) if args.steps else 0,
        "gpu_launches_total": int(launches), "served": None,
    }
    if not args.no_serve and world == 1:
        result["served"] = run_served(torch, cs, dev, args.serve_requests, loads=(0.25, 0.5, 0.75, 0.9))
        result["mppi"] = run_mppi(torch, cs, dev)
        result["rrt"] = run_rrt(torch, cs, dev)
        result["refine"] = run_refine(torch, cs, dev)
        result["variants"] = run_variants(torch, cs, dev)
        result["render"] = run_render(torch, cs, dev)
    return result


def run_e2e(args, cs, torch, dev, stream, scene_h, arm_h, edge_h, poses_h, offs_h, radius,
            useful_pairs, world, tiles):
    """The same step end to end through the C ABI from pinned host memory:
    the scene built from host arrays (the library copies them in), the step's
    query batches copied in once on a second stream while the scene is
    built, the same queries as the device-timed step
    (same tile shapes) on device buffers, and every pass's outputs copied back
    to pinned host memory on a second stream while the next pass computes."""
    import ctypes

    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h_scene = {k: pin(v) for k, v in scene_h.items()}
    h_arm, h_edge, h_poses = pin(arm_h), pin(edge_h), pin(poses_h)
    d_offs = torch.as_tensor(offs_h, device=dev)
    K = offs_h.shape[0]
    n_pose = poses_h.shape[0]
    copy = torch.cuda.Stream(dev)
    sizes = [(len(NSIGMAS) * h_arm.shape[0], 64), (len(NSIGMAS) * h_edge.shape[0], 1024)]
    dev_out, host_out = [], []
    for Q, G in sizes:
        ng = (Q + G - 1) // G
        dev_out.append({"metric": torch.empty(Q, device=dev), "collide": torch.empty(Q, dtype=torch.uint8, device=dev),
                        "group_metric": torch.empty(ng, device=dev),
                        "group_collide": torch.empty(ng, dtype=torch.uint8, device=dev)})
        host_out.append({k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in dev_out[-1].items()})
    h_gpose = torch.empty((n_pose, 6)).pin_memory()
    h_posecost = torch.empty(n_pose).pin_memory()
    h2d = sum(v.numel() * 4 for v in h_scene.values()) + (h_arm.numel() + h_edge.numel() + h_poses.numel()) * 4
    d2h = sum(v.numel() * v.element_size() for o in host_out for v in o.values()) \
        + h_gpose.numel() * 4 + h_posecost.numel() * 4
    sh = stream.cuda_stream

    def step():
        # the query batches travel on the copy stream while the scene is built
        with torch.cuda.stream(copy):
            d_arm = h_arm.to(dev, non_blocking=True)
            d_edge = h_edge.to(dev, non_blocking=True)
            d_poses = h_poses.to(dev, non_blocking=True)
        for t in (d_arm, d_edge, d_poses):
            t.record_stream(stream)
        uploaded = torch.cuda.Event()
        uploaded.record(copy)
        d = cs.abi.cs_scene_desc()
        d.n = scene_h["means"].shape[0]
        d.means, d.scales = h_scene["means"].data_ptr(), h_scene["scales"].data_ptr()
        d.quats, d.opacity = h_scene["quats"].data_ptr(), h_scene["opacity"].data_ptr()
        d.on_device, d.use_filter, d.opacity_min, d.extent_max = 0, 1, 0.05, 0.1
        h = ctypes.c_void_p()
        cs.check(cs.abi.cs_scene_create(d, sh, h))
        stream.wait_event(uploaded)
        for i, (name, dq, G) in enumerate((("arm", d_arm, 64), ("edge", d_edge, 1024))):
            o = dev_out[i]
            p = cs.QueryParams(group_size=G, tile_config=tiles[name], sweep=NSIGMAS).to_c()
            p.stream = sh
            p.out_group_metric, p.out_group_collide = o["group_metric"].data_ptr(), o["group_collide"].data_ptr()
            cs.check(cs.abi.cs_query(h, 0, dq, dq.shape[0], 0.0, o["metric"], o["collide"], p))
            done = torch.cuda.Event()
            done.record(stream)
            copy.wait_event(done)
            with torch.cuda.stream(copy):
                for k, v in o.items():
                    host_out[i][k].copy_(v, non_blocking=True)
        with torch.cuda.stream(stream):
            sph = cs.pose_spheres(d_poses, d_offs, radius, stream=stream)
            Q = sph.shape[0]
            # forward (the per-pose cost) and adjoint in one fused launch
            p = cs.QueryParams(group_size=K).to_c()
            p.stream = sh
            gm = torch.empty(n_pose, device=dev)
            p.out_group_metric = gm.data_ptr()
            g = torch.empty((Q, 3), device=dev)
            ones = torch.ones(n_pose, device=dev)
            cs.check(cs.abi.cs_query_fwd_grad(h, 0, sph, Q, 1.0, ones, None, None, g, p))
            gp = cs.pose_spheres_grad(d_poses, d_offs, g, stream=stream)
            h_gpose.copy_(gp, non_blocking=True)
            h_posecost.copy_(gm, non_blocking=True)
        stream.synchronize()
        copy.synchronize()
        cs.check(cs.abi.cs_scene_destroy(h))

    for _ in range(max(1, args.warmup)):
        step()
    times = []
    for _ in range(args.steps):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        step()
        times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    return {"value": world * useful_pairs / (ms * 1e-3), "unit": "pairs/s", "ms_per_step": ms,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "note": "scene built from pinned host arrays, query batches copied in once per step on a second "
                    "stream while the scene is built, outputs copied back per pass on that stream; same tile "
                    "shapes as the device-timed step"}


# ------------------------------------------------------------ serving
SERVE_WORKLOAD = ("2 apartment scenes x 3M Gaussians; Poisson requests of 16..262,144 spheres "
                  "(log-uniform), n_sigma ~ U[0,2], scene ~ U{0,1}")


def _pct(xs, q):
    return float(np.percentile(np.asarray(xs), q)) if len(xs) else None


def serve_setup(torch, cs, dev):
    import cs_synth as S
    scenes_h = [S.apartment_scene(seed=1005), S.apartment_scene(seed=1006)]
    scenes = [cs.Scene(s["means"], s["scales"], s["quats"], s["opacity"], device=dev) for s in scenes_h]
    # tile shape per scene from the autotuner, on a full-size request mix
    # tile shapes per batch-size class from the autotuner, on request mixes
    tune = S.serving_requests(seed=1999, count=48, q_lo=16, q_hi=262_144)
    rows = np.concatenate([r["spheres"] for r in tune])
    tiles = []
    for sc in scenes:
        per = {}
        for lg in (9, 12, 15, 17, 19):
            batch = torch.as_tensor(rows[: 1 << lg], device=dev)
            per[1 << lg] = sc.autotune(batch, 1.0, reps=2)[0]
        tiles.append(per)
    torch.cuda.synchronize(dev)
    return scenes_h, scenes, tiles


def served_burst(cs, server, reqs):
    """All requests submitted at once: the served capacity (rows/s)."""
    t0 = server.clock()
    ts = [server.submit(r["scene"], r["spheres"], r["nsigma"]) for r in reqs]
    last = t0
    for t in ts:
        _, tm = server.wait(t, timeout=600.0)
        last = max(last, tm["completed"])
    rows = sum(r["spheres"].shape[0] for r in reqs)
    return rows / (last - t0), last - t0


def served_poisson(cs, server, reqs, rate_rows_s):
    """Requests submitted at Poisson arrival times scaled to `rate_rows_s`
    offered rows/s; latency = completion - intended arrival."""
    rows = np.array([r["spheres"].shape[0] for r in reqs], np.float64)
    arr = np.array([r["arrival"] for r in reqs])
    arr = arr * (rows.mean() / rate_rows_s) / max(np.diff(arr).mean(), 1e-12)
    tickets = [None] * len(reqs)
    t0 = server.clock() + 0.05

    def client():
        for k, r in enumerate(reqs):
            while True:
                dt = t0 + arr[k] - server.clock()
                if dt <= 0:
                    break
                time.sleep(min(dt, 0.002) if dt > 0.0005 else 0)
            tickets[k] = server.submit(r["scene"], r["spheres"], r["nsigma"])

    th = threading.Thread(target=client)
    th.start()
    lat, done_last = [], t0
    for k in range(len(reqs)):
        while tickets[k] is None:
            time.sleep(0.0002)
        _, tm = server.wait(tickets[k], timeout=600.0)
        lat.append(tm["completed"] - (t0 + arr[k]))
        done_last = max(done_last, tm["completed"])
    th.join()
    span = done_last - t0
    return {"offered_rows_per_s": rate_rows_s, "p50_ms": 1e3 * _pct(lat, 50), "p99_ms": 1e3 * _pct(lat, 99),
            "mean_ms": 1e3 * float(np.mean(lat)), "queries_per_s": float(rows.sum() / span),
            "requests": len(reqs)}


def per_call_run(cs, scenes, reqs, rate_rows_s=None):
    """The plain per-call path: one cs_query call per request (host buffers,
    copies in, compute, copies out, synchronise), serially in arrival order.
    rate None: back to back (capacity); else Poisson arrivals at that rate."""
    rows = np.array([r["spheres"].shape[0] for r in reqs], np.float64)
    arr = np.array([r["arrival"] for r in reqs])
    if rate_rows_s is not None:
        arr = arr * (rows.mean() / rate_rows_s) / max(np.diff(arr).mean(), 1e-12)
    lat = []
    t0 = time.perf_counter() + 0.01
    for k, r in enumerate(reqs):
        if rate_rows_s is not None:
            while time.perf_counter() < t0 + arr[k]:
                time.sleep(0.0002)
        q = r["spheres"]
        m = np.empty(q.shape[0], np.float32)
        c = np.empty(q.shape[0], np.uint8)
        p = cs.QueryParams().to_c()
        p.host_io = 1
        cs.check(cs.abi.cs_query(scenes[r["scene"]].handle, 0, q, q.shape[0], r["nsigma"], m, c, p))
        done = time.perf_counter()
        lat.append(done - (t0 + (arr[k] if rate_rows_s is not None else 0.0)))
    span = time.perf_counter() - t0
    out = {"queries_per_s": float(rows.sum() / span), "requests": len(reqs)}
    if rate_rows_s is not None:
        out.update({"offered_rows_per_s": rate_rows_s, "p50_ms": 1e3 * _pct(lat, 50),
                    "p99_ms": 1e3 * _pct(lat, 99), "mean_ms": 1e3 * float(np.mean(lat))})
    return out


def one_query_per_call(cs, torch, scene, n=2000):
    """One sphere per cs_query call (device buffers, synchronised): the
    launch-bound floor of a per-query interface."""
    import cs_synth as S
    q = torch.as_tensor(S.serving_requests(seed=1998, count=1, q_lo=n, q_hi=n + 1)[0]["spheres"][:n],
                        device="cuda")
    m = torch.empty(1, device="cuda")
    c = torch.empty(1, dtype=torch.uint8, device="cuda")
    for j in range(20):
        scene.query(q[j:j + 1], 1.0, out={"metric": m, "collide": c})
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for j in range(n):
        scene.query(q[j:j + 1], 1.0, out={"metric": m, "collide": c})
        torch.cuda.synchronize()
    return n / (time.perf_counter() - t0)


def run_served(torch, cs, dev, n_requests, loads=(0.75,), with_per_call=True, slots=3, slot_rows=1 << 19,
               use_graphs=True):
    import cs_synth as S
    scenes_h, scenes, tiles = serve_setup(torch, cs, dev)
    reqs = S.serving_requests(seed=1007, count=n_requests)
    warm = S.serving_requests(seed=1008, count=16, q_lo=16, q_hi=65536)
    srv = cs.Server(scenes, slots=slots, slot_rows=slot_rows, tile_config=cs.abi.CS_TILE_TUNED,
                    use_graphs=use_graphs)
    served_burst(cs, srv, warm)
    if use_graphs:  # capture every (scene, size bucket) graph before timing
        served_burst(cs, srv, [dict(r, scene=s) for s in range(len(scenes))
                               for r in S.serving_requests(seed=1009, count=12, q_lo=512, q_hi=1 << 19)])
    cap, cap_s = served_burst(cs, srv, reqs)
    runs = [served_poisson(cs, srv, reqs, f * cap) for f in loads]
    st = srv.stats()
    srv.close()
    out = {"workload": SERVE_WORKLOAD, "requests": n_requests,
           "rows": int(sum(r["spheres"].shape[0] for r in reqs)),
           "served_capacity_queries_per_s": cap, "loads": [dict(r, load=f) for f, r in zip(loads, runs)],
           "server": {"slots": slots, "slot_rows": slot_rows, "tiles": tiles, "graphs": bool(use_graphs),
                      "mean_batch_requests": st["requests"] / max(st["batches"], 1),
                      "max_batch_requests": st["max_batch_requests"]}}
    if with_per_call:
        per_call_run(cs, scenes, warm)
        pc_cap = per_call_run(cs, scenes, reqs)
        out["per_call"] = {"capacity_queries_per_s": pc_cap["queries_per_s"],
                           "loads": [dict(per_call_run(cs, scenes, reqs, f * cap), load=f) for f in loads[:1]]}
        out["one_query_per_call_queries_per_s"] = one_query_per_call(cs, torch, scenes[0])
    for sc in scenes:
        sc.close()
    return out


def run_build_case(args, reps=10):
    """The scene build alone (cs_scene_create from device arrays: Eq. 2
    repack, floater filter, Hilbert order, chunks, tree) on the 1M tabletop,
    `reps` times after two warm-up builds; CUDA events on the build's stream
    (the call returns with the scene complete)."""
    import torch

    import cs_synth as S
    import paper_2609_35619_b300 as cs
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    sc = S.tabletop_scene()
    d = {k: torch.as_tensor(v, device=dev) for k, v in sc.items()}
    stream = torch.cuda.Stream(dev)
    ms = []
    for r in range(reps + 2):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        scene = cs.Scene(d["means"], d["scales"], d["quats"], d["opacity"], device=dev, stream=stream)
        e1.record(stream)
        e1.synchronize()
        if r >= 2:
            ms.append(e0.elapsed_time(e1))
        scene.close()
    n = sc["means"].shape[0]
    print(json.dumps({"case": "build", "gaussians": n, "ms_mean": float(np.mean(ms)), "ms_min": float(np.min(ms)),
                      "algorithmic_gbs": n * 84 / (np.min(ms) * 1e-3) / 1e9}))


def run_serve_case(args):
    import torch

    import paper_2609_35619_b300 as cs
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    res = run_served(torch, cs, dev, args.serve_requests_sweep, loads=(0.25, 0.5, 0.75, 0.9),
                     with_per_call=not args.no_per_call, slots=args.serve_slots, slot_rows=args.serve_rows,
                     use_graphs=not args.serve_eager)
    print(json.dumps({"case": "serve", **res}))


# --------------------------------------------------------------- MPPI
MPPI_WORKLOAD = "drone room 500k Gaussians; MPPI iteration with 1,024 rollouts x 32 steps x 1 sphere (r = 0.15 m)"


def run_mppi(torch, cs, dev, iters=20, K=1024, T=32, with_oracle=False):
    """One MPPI iteration (rollouts, metric, costs, Eq. 10 weights, update)
    timed with CUDA events over `iters` back-to-back iterations, each
    starting from the previous nominal sequence, inputs resident on the device."""
    import cs_synth as S
    sc = S.drone_scene()
    scene = cs.Scene(sc["means"], sc["scales"], sc["quats"], sc["opacity"], device=dev)
    rng = np.random.default_rng(1002)
    x0 = torch.tensor([3.0, 2.5, 1.5], device=dev)
    U = torch.as_tensor(np.tile([0.4, -0.2, 0.05], (T, 1)).astype(np.float32), device=dev)
    eps = torch.as_tensor(rng.normal(0, 0.6, (iters + 3, K, T, 3)).astype(np.float32), device=dev)
    out = {"U": torch.empty((T, 3), device=dev), "cost": torch.empty(K, device=dev),
           "weights": torch.empty(K, device=dev), "collide": torch.empty(K, dtype=torch.uint8, device=dev)}
    kw = dict(dt=0.1, radius=0.15, nsigma=1.0, lam=1.0, goal=(4.5, 1.0, 1.25))
    eps_buf = torch.empty_like(eps[0])

    def timed(one_iteration):
        for i in range(3):
            eps_buf.copy_(eps[i])
            one_iteration()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = cs.abi.cs_launch_count()
        e0.record()
        for i in range(iters):
            eps_buf.copy_(eps[3 + i])
            one_iteration()
        e1.record()
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / iters, (cs.abi.cs_launch_count() - l0) / iters

    U0 = U.clone()

    def eager():
        cs.mppi_step(scene, x0, U, eps_buf, out=out, **kw)
        U.copy_(out["U"])

    ms, kernels = timed(eager)
    U.copy_(U0)
    graph = cs.MppiGraph(scene, x0, U, eps_buf, in_place=True, **kw)
    ms_graph, _ = timed(graph.launch)
    res = {"workload": MPPI_WORKLOAD, "K": K, "T": T, "ms_per_iteration": ms, "iterations_per_s": 1e3 / ms,
           "queries_per_s": K * T * 1e3 / ms, "kernels_per_iteration": kernels,
           "graph_ms_per_iteration": ms_graph, "graph_iterations_per_s": 1e3 / ms_graph,
           "mean_cost": float(graph.out["cost"].mean()), "collide_frac": float(graph.out["collide"].float().mean()),
           "note": "each iteration also copies its perturbations into the buffer the call reads"}
    graph.close()
    scene.close()
    return res


RRT_WORKLOAD = ("drone room 500k Gaussians; batched RRT extensions of 32 samples, 8 checked points per edge, "
                "sphere r = 0.05 m, step 0.3 m, n_sigma 1")


def run_rrt(torch, cs, dev, iters=200, B=32, M=8):
    """Batched RRT from the room centre: `iters` extensions (nearest, steer,
    flags-mode edge check with early exit, insertion), timed with CUDA events
    back to back, samples resident on the device."""
    import cs_synth as S
    sc = S.drone_scene()
    scene = cs.Scene(sc["means"], sc["scales"], sc["quats"], sc["opacity"], device=dev)
    rng = np.random.default_rng(1010)
    samples = torch.as_tensor(rng.uniform([0.1, 0.1, 0.1], [5.9, 4.9, 2.9], (iters + 5, B, 3)).astype(np.float32),
                              device=dev)
    tree = cs.RrtTree(scene, [3.0, 2.5, 1.5], capacity=1 << 16, step=0.3, radius=0.05, nsigma=1.0, M=M)
    for i in range(5):
        tree.extend(samples[i])
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n0 = int(tree.count.item())
    l0 = cs.abi.cs_launch_count()
    e0.record()
    for i in range(iters):
        tree.extend(samples[5 + i])
    e1.record()
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / iters
    k_ext = (cs.abi.cs_launch_count() - l0) / iters
    n1 = int(tree.count.item())
    # the same loop through a captured extension: samples written into the
    # graph's buffer on the stream, then one graph launch per extension
    gtree = cs.RrtTree(scene, [3.0, 2.5, 1.5], capacity=1 << 16, step=0.3, radius=0.05, nsigma=1.0, M=M)
    g = gtree.graph(B)
    for i in range(5):
        g.samples.copy_(samples[i])
        g.launch()
    torch.cuda.synchronize(dev)
    e0.record()
    for i in range(iters):
        g.samples.copy_(samples[5 + i])
        g.launch()
    e1.record()
    torch.cuda.synchronize(dev)
    g_ms = e0.elapsed_time(e1) / iters
    same = int(gtree.count.item()) == n1
    g.close()
    res = {"workload": RRT_WORKLOAD, "B": B, "M": M, "extensions": iters, "ms_per_extension": ms,
           "graph_ms_per_extension": g_ms, "graph_edges_per_s": B * 1e3 / g_ms, "graph_same_tree_size": same,
           "edges_per_s": B * 1e3 / ms, "points_per_s": B * M * 1e3 / ms,
           "kernels_per_extension": k_ext,
           "nodes_before": n0, "nodes_after": n1, "free_frac": (n1 - n0) / (B * iters)}
    scene.close()
    return res


def run_variants(torch, cs, dev, iters=5):
    """Variants of the metric on the 1M tabletop, each one launch per call at
    n_sigma 1 with the default tile shape, the fused kernel timed with CUDA
    events (mean of `iters` calls after two warm-up calls): Gaussians as
    printed (Eq. 7), the exact-variance option, the scene as 2DGS disks and as
    a point cloud (262,144 arm spheres each), and the arm as 229,376 link
    ellipsoids (with Eq. 7 and the exact variance)."""
    import cs_synth as S
    arm = torch.as_tensor(S.arm_queries(), device=dev)
    ell = torch.as_tensor(S.arm_ellipsoids(), device=dev)
    cases = [("gaussians", "tabletop", arm, 0, 64, False), ("exact_variance", "tabletop", arm, 0, 64, True),
             ("disks_2dgs", "disks", arm, 0, 64, False), ("point_cloud", "points", arm, 0, 64, False),
             ("ellipsoid_arm", "tabletop", ell, 1, 7, False),
             ("ellipsoid_arm_exact_variance", "tabletop", ell, 1, 7, True)]
    gens = {"tabletop": S.tabletop_scene, "disks": S.tabletop_disks, "points": S.tabletop_points}
    scenes, out = {}, {}
    for name, kind, q, prim, G, exact in cases:
        if kind not in scenes:
            sc = gens[kind]()
            scenes[kind] = cs.Scene(sc["means"], sc["scales"], sc["quats"], sc["opacity"], device=dev)
        scene = scenes[kind]
        qp = cs.QueryParams(group_size=G, exact_variance=exact)
        for _ in range(2):
            scene.query(q, 1.0, prim_type=prim, params=qp)
        stats = torch.zeros(2, dtype=torch.int64, device=dev)
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(iters)]
        for i in range(iters):
            scene.query(q, 1.0, prim_type=prim, params=qp, pair_stats=stats, eval_events=evs[i])
        torch.cuda.synchronize(dev)
        ms = sum(a.elapsed_time(b) for a, b in evs) / iters
        cand, useful = (v // iters for v in stats.cpu().tolist())
        out[name] = {"rows": int(q.shape[0]), "prim": "ellipsoid" if prim else "sphere", "eval_ms": ms,
                     "useful_pairs": useful, "candidate_pairs": cand, "useful_pairs_per_s": useful / (ms * 1e-3)}
    for scene in scenes.values():
        scene.close()
    return {"workload": "tabletop 1M (as printed / 2DGS disks / point cloud); 262,144 arm spheres or "
                        "229,376 link ellipsoids; n_sigma 1; default tile shapes", **out}


RENDER_WORKLOAD = ("drone room 500k Gaussians; the terminal states of 256 MPPI rollouts rendered at "
                   "128 x 128 (near plane 0.2 m), RGB + depth + alpha, one call per batch")


def run_render(torch, cs, dev, iters=10, views=256, width=128, height=128):
    """Batched image synthesis (Eq. 3-4): `views` terminal-state images of
    the drone room per call, timed with CUDA events on the stream around each
    call (the call waits for the stream once, mid-way, to size its instance
    list), after two warm-up calls."""
    import cs_synth as S
    sc = S.drone_scene()
    scene = cs.Scene(sc["means"], sc["scales"], sc["quats"], sc["opacity"], device=dev)
    scene.set_appearance(sc["opacity"], S.scene_colors(sc))
    cams = torch.as_tensor(S.drone_terminal_cameras(rollouts=views, width=width, height=height), device=dev)
    out = None
    for _ in range(2):
        out = scene.render(cams, width, height, near_plane=0.2, out=out)
    torch.cuda.synchronize(dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(iters)]
    l0 = cs.abi.cs_launch_count()
    for a, b in evs:
        a.record()
        scene.render(cams, width, height, near_plane=0.2, out=out)
        b.record()
    torch.cuda.synchronize(dev)
    ms = sorted(a.elapsed_time(b) for a, b in evs)
    med = ms[len(ms) // 2]
    res = {"workload": RENDER_WORKLOAD, "views": views, "width": width, "height": height,
           "ms_per_call": med, "ms_min": ms[0], "images_per_s": views * 1e3 / med,
           "pixels_per_s": views * width * height * 1e3 / med,
           "kernels_per_call": (cs.abi.cs_launch_count() - l0) / iters,
           "instances": scene.last_render_instances,
           "mean_alpha": float(out["alpha"].mean().item())}
    scene.close()
    return res


REFINE_WORKLOAD = ("drone room 500k Gaussians; one zeroth-order refinement step of a 32-control-point plan "
                   "across the room: 1,024 perturbed B-splines x 8 samples per segment (270,336 spheres, "
                   "r = 0.1 m, n_sigma 1)")


def run_refine(torch, cs, dev, iters=20, K=1024, N=32, M=8):
    """Zeroth-order path refinement (one MPPI step over the plan's B-spline
    control points), timed with CUDA events over `iters` back-to-back steps,
    inputs resident on the device."""
    import cs_synth as S
    sc = S.drone_scene()
    scene = cs.Scene(sc["means"], sc["scales"], sc["quats"], sc["opacity"], device=dev)
    rng = np.random.default_rng(1012)
    a, b = np.array([0.8, 0.7, 1.2]), np.array([5.2, 4.3, 1.6])
    t = np.linspace(0, 1, N)[:, None]
    P = (a + t * (b - a) + np.r_[np.zeros((1, 3)), rng.normal(0, 0.2, (N - 2, 3)), np.zeros((1, 3))])
    ctrl = torch.as_tensor(P.astype(np.float32), device=dev)
    eps = torch.as_tensor(rng.normal(0, 0.1, (K, N, 3)).astype(np.float32), device=dev)
    out = None
    for _ in range(3):
        out = cs.path_refine(scene, ctrl, eps, M=M, radius=0.1, out=out)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = cs.abi.cs_launch_count()
    e0.record()
    for _ in range(iters):
        cs.path_refine(scene, ctrl, eps, M=M, radius=0.1, out=out)
    e1.record()
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / iters
    P_pts = (N + 1) * M + 1
    res = {"workload": REFINE_WORKLOAD, "K": K, "N": N, "M": M, "ms_per_step": ms,
           "samples_per_s": K * P_pts * 1e3 / ms,
           "kernels_per_step": (cs.abi.cs_launch_count() - l0) / iters}
    scene.close()
    return res


def run_rrt_case(args):
    import torch

    import paper_2609_35619_b300 as cs
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    print(json.dumps({"case": "rrt", **run_rrt(torch, cs, dev)}))


def run_mppi_case(args):
    import torch

    import paper_2609_35619_b300 as cs
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    print(json.dumps({"case": "mppi", **run_mppi(torch, cs, dev, iters=max(args.steps, 1) * 10)}))


# ------------------------------------------------------------- oracle
def oracle_sample(target_s: float, seed: int = 0):
    """Time the FP64 oracle on a bounded sample of the workload: rows drawn
    from the arm and edge batches (half each) at n_sigma = 1 against the full
    scene, sized to about target_s seconds of host time."""
    import oracle
    scene, arm, edge, poses, offs, radius = make_inputs()
    rng = np.random.default_rng(seed)
    probe = np.concatenate([arm[rng.choice(arm.shape[0], 32)], edge[rng.choice(edge.shape[0], 32)]])
    oracle.query(scene, probe[:2], 0, 1.0)  # thread pool start-up
    t0 = time.perf_counter()
    oracle.query(scene, probe, 0, 1.0)
    per_row = (time.perf_counter() - t0) / probe.shape[0]
    rows = int(max(4, min(65536, target_s / max(per_row, 1e-7))))
    rows -= rows % 2
    sample = np.concatenate([arm[rng.choice(arm.shape[0], rows // 2, replace=False)],
                             edge[rng.choice(edge.shape[0], rows // 2, replace=False)]])
    t0 = time.perf_counter()
    res = oracle.query(scene, sample, 0, 1.0)
    dt = time.perf_counter() - t0
    if dt < 0.5 * target_s and rows < 65536:  # the probe overestimated the cost of a row: once more, larger
        rows = int(min(65536, rows * target_s / max(dt, 1e-3)))
        rows -= rows % 2
        sample = np.concatenate([arm[rng.choice(arm.shape[0], rows // 2, replace=False)],
                                 edge[rng.choice(edge.shape[0], rows // 2, replace=False)]])
        t0 = time.perf_counter()
        res = oracle.query(scene, sample, 0, 1.0)
        dt = time.perf_counter() - t0
    useful = int(res["count_nbr"].sum())
    n = scene["means"].shape[0]
    # the parity checks' exclusions and widened bounds on these rows (the
    # oracle's diagnostics; the contract in tests/_parity.py): rows in the
    # cutoff band, in the collision band, and cost rows whose Eq. 8 cancels
    # strongly enough to take the derived bound instead of 1e-5
    cut = res["band_cut"] > 0
    parity = {"rows": rows, "cutoff_band_rows": int(cut.sum()), "collision_band_rows": int((res["band_in"] > 0).sum()),
              "widened_rows": int(((res["cond_cost"] > 50.0) & ~cut).sum())}
    return {"value": useful / dt, "unit": "pairs/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{rows} rows (half arm, half edge spheres) at n_sigma=1 against all {n} Gaussians; "
                      f"{useful} useful pairs, {rows * n} dense pairs in {dt:.2f} s "
                      f"({rows * n / dt:.3g} dense pairs/s)",
            "parity_sample": parity, "seconds": dt}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    vals = []
    for _ in range(args.warmup):
        oracle_sample(2.0, seed=99)
    per_step = max(5.0, 120.0 / max(args.steps, 1))
    for k in range(args.steps):
        vals.append(oracle_sample(per_step, seed=k))
    value = statistics.mean(v["value"] for v in vals)
    ms = 1e3 * statistics.mean(v["seconds"] for v in vals)
    last = vals[-1]
    return {"impl": "reference", "metric": "query-Gaussian pair evals/s (useful pairs inside the neighbour sets)",
            "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + " (bounded sample per step)", "parallelism": "host cores"},
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": last["cores"], "kind": "oracle",
                             "sample": last["sample"]},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_eval_case(args):
    """Small case for kernel profiles: one scene build and two launches of the
    fused kernel over the 262,144 arm spheres (the second is the measured one;
    a third, untimed, reads the kernel counters)."""
    import torch

    import cs_synth as S
    import paper_2609_35619_b300 as cs
    dev = torch.device("cuda", 0)
    sc = S.tabletop_scene()
    batches = {"arm": S.arm_queries, "edge": S.edge_queries, "arm_ellipsoids": S.arm_ellipsoids}
    arm = torch.as_tensor(batches[args.batch](), device=dev)
    scene = cs.Scene(sc["means"], sc["scales"], sc["quats"], sc["opacity"], device=dev, cell_size=args.cell)
    G = {"arm": 64, "edge": 1024, "arm_ellipsoids": 7}[args.batch]
    prim = cs.CS_PRIM_ELLIPSOID if args.batch == "arm_ellipsoids" else cs.CS_PRIM_SPHERE
    qp = cs.QueryParams(group_size=G, tile_config=args.tile, exact_variance=args.exact,
                        mode=cs.CS_METRIC_FLAGS if args.flags else cs.CS_METRIC_MEAN_COST)
    ns = args.nsigma
    stats = torch.zeros(2, dtype=torch.int64, device=dev)
    kstats = torch.zeros(16, dtype=torch.int64, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    if args.sweep:
        # one launch over the four n_sigma values (cs_params sweep) against four launches
        Q = arm.shape[0]
        qs = cs.QueryParams(group_size=G, tile_config=args.tile, sweep=tuple(NSIGMAS))
        ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        for _ in range(2):
            o1 = scene.query(arm, 0.0, params=qs, prim_type=prim)
        scene.query(arm, 0.0, params=qs, prim_type=prim, eval_events=ev1, out=o1)
        scene.query(arm, 0.0, params=qs, prim_type=prim, kernel_stats=kstats)
        sep_ms = 0.0
        outs = []
        for ns in NSIGMAS:
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            scene.query(arm, ns, params=qp, prim_type=prim)
            o = scene.query(arm, ns, params=qp, prim_type=prim, eval_events=ev)
            torch.cuda.synchronize()
            sep_ms += ev[0].elapsed_time(ev[1])
            outs.append(o["metric"].clone())
        torch.cuda.synchronize()
        same = all(torch.equal(o1["metric"][i * Q:(i + 1) * Q], outs[i]) for i in range(len(NSIGMAS)))
        ks = kstats.cpu().tolist()
        print(json.dumps({"case": "eval", "sweep": True, "batch": args.batch, "tile": args.tile,
                          "queries": 4 * Q, "one_launch_ms": ev1[0].elapsed_time(ev1[1]),
                          "four_launches_ms": sep_ms, "bitwise_equal": bool(same),
                          "consumer_wait_frac": ks[9] / max(ks[8], 1), "producer_wait_frac": ks[11] / max(ks[10], 1),
                          "kernel_stats": dict(zip(KSTAT_NAMES, ks))}))
        return
    if args.grad:
        up = torch.ones(arm.shape[0] // G + (arm.shape[0] % G > 0), device=dev)
        if args.fused:
            fp = cs.QueryParams(group_size=G)
            scene.query_fwd_grad(arm, ns, grad_out=up, params=fp)
            scene.query_fwd_grad(arm, ns, grad_out=up, params=fp, eval_events=ev)
            torch.cuda.synchronize()
            print(json.dumps({"case": "eval", "grad": True, "fused": True, "batch": args.batch, "nsigma": ns,
                              "queries": arm.shape[0], "eval_ms": ev[0].elapsed_time(ev[1])}))
            return
        scene.query_grad(arm, ns, grad_out=up, params=qp, prim_type=prim)
        scene.query_grad(arm, ns, grad_out=up, params=qp, eval_events=ev, prim_type=prim)
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1])
        print(json.dumps({"case": "eval", "grad": True, "batch": args.batch, "tile": args.tile, "nsigma": ns,
                          "exact": args.exact, "queries": arm.shape[0], "eval_ms": ms}))
        return
    scene.query(arm, ns, params=qp, prim_type=prim)
    scene.query(arm, ns, params=qp, pair_stats=stats, eval_events=ev, prim_type=prim)
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1])
    scene.query(arm, ns, params=qp, kernel_stats=kstats, prim_type=prim)
    torch.cuda.synchronize()
    scene.sync()
    cand, useful = stats.cpu().tolist()
    names = KSTAT_NAMES
    print(json.dumps({"case": "eval", "batch": args.batch, "tile": args.tile, "nsigma": ns,
                      "exact": args.exact, "flags": args.flags, "queries": arm.shape[0], "useful_pairs": useful,
                      "candidate_pairs": cand, "eval_ms": ms,
                      "kernel_stats": dict(zip(names, kstats.cpu().tolist())), "info": scene.info()}))


def main():
    args = parse()
    if args.case == "eval":
        run_eval_case(args)
        return
    if args.case == "build":
        return run_build_case(args)
    if args.case == "serve":
        run_serve_case(args)
        return
    if args.case == "mppi":
        run_mppi_case(args)
        return
    if args.case == "render":
        import torch

        import paper_2609_35619_b300 as cs
        dev = torch.device("cuda", 0)
        torch.cuda.set_device(dev)
        print(json.dumps({"case": "render", **run_render(torch, cs, dev, iters=max(args.steps, 1))}))
        return
    if args.case == "variants":
        import torch

        import paper_2609_35619_b300 as cs
        dev = torch.device("cuda", 0)
        torch.cuda.set_device(dev)
        print(json.dumps({"case": "variants", **run_variants(torch, cs, dev)}))
        return
    if args.case == "rrt":
        run_rrt_case(args)
        return
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if world > 1 and args.impl == "ours":
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        out = run_ours(args, rank, world)
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            cb = oracle_sample(15.0)
            cb.pop("seconds", None)
            out["cpu_baseline"] = cb
    if rank == 0 and out is not None:
        print(json.dumps(out))
    if world > 1 and args.impl == "ours":
        import torch.distributed as tdist
        tdist.destroy_process_group()


if __name__ == "__main__":
    main()
