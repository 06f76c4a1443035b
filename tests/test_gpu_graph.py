"""Captured query graphs and the tile autotuner, through the C ABI.

A graph replays exactly the launches of the call it captured, so its
outputs must equal that call's bit for bit, also after the primitives are
rewritten in place; the autotuner must return one of the listed shapes and a
CS_TILE_TUNED call must equal a call with the shape it chose (every shape
computes the same bits: each lane reduces a fixed subsequence of the
Gaussians in a fixed order, whatever the tile).
"""
import numpy as np
import pytest

import cs_synth as S
import oracle
from _parity import compare, to_np

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cs(cuda_device):
    import paper_2609_35619_b300 as cs
    return cs


@pytest.fixture(scope="module")
def table(cs):
    sc = S.tabletop_scene(n=200_000)
    return sc, cs.Scene(sc["means"], sc["scales"], sc["quats"], sc["opacity"])


def _same(a, b, keys):
    for k in keys:
        np.testing.assert_array_equal(a[k].cpu().numpy(), b[k].cpu().numpy(), err_msg=k)


def test_every_tile_shape_gives_the_same_bits(cs, table):
    sc, scene = table
    q = torch.as_tensor(S.arm_queries(configs=64), device="cuda")
    ref = None
    for t in cs.abi.cs_tile_configs():
        for mode in (0, 2, 3):
            out = scene.query(q, 1.0, params=cs.QueryParams(mode=mode, tile_config=t), want_count=True)
            torch.cuda.synchronize()
            if t == 1:
                ref = ref or {}
                ref[mode] = {k: v.clone() for k, v in out.items()}
            else:
                _same(out, ref[mode], ["metric", "collide", "count"])


def test_forward_graph_replays_the_call(cs, table):
    sc, scene = table
    rng = np.random.default_rng(11)
    q0 = S.arm_queries(configs=48)
    prims = torch.as_tensor(q0, device="cuda").contiguous()
    params = cs.QueryParams(group_size=64)
    g = cs.QueryGraph(scene, prims, 1.0, params=params, want_count=True)
    assert g.kernels > 3
    n0 = cs.abi.cs_launch_count()
    out = g.launch()
    g.sync()
    assert cs.abi.cs_launch_count() - n0 == g.kernels
    ref = scene.query(prims, 1.0, params=params, want_count=True)
    torch.cuda.synchronize()
    _same(out, ref, ["metric", "collide", "count", "group_metric", "group_collide"])
    # new primitives written in place; the same graph answers for them
    q1 = q0.copy()
    q1[:, :3] += rng.normal(0, 0.02, (q1.shape[0], 3)).astype(np.float32)
    prims.copy_(torch.as_tensor(q1))
    g.launch()
    g.sync()
    ref1 = scene.query(torch.as_tensor(q1, device="cuda"), 1.0, params=params, want_count=True)
    torch.cuda.synchronize()
    _same(g.out, ref1, ["metric", "collide", "count", "group_metric", "group_collide"])
    # and both agree with the oracle on a sample of rows
    rows = rng.choice(q1.shape[0], 256, replace=False)
    sub = {k: g.out[k].cpu().numpy()[rows] for k in ("metric", "collide", "count")}
    compare(sub, oracle.query(sc, q1[rows], 0, 1.0), 0, oracle.Params(), "graph replay")
    g.close()


def test_adjoint_graph_and_concurrent_graphs(cs, table):
    sc, scene = table
    qa = torch.as_tensor(S.arm_queries(configs=32), device="cuda").contiguous()
    qb = torch.as_tensor(S.arm_queries(configs=40, seed=5), device="cuda").contiguous()
    up = torch.as_tensor(np.random.default_rng(2).normal(size=qa.shape[0]).astype(np.float32), device="cuda")
    ga = cs.QueryGraph(scene, qa, 1.0, grad=True, grad_out=up)
    gb = cs.QueryGraph(scene, qb, 0.5, params=cs.QueryParams(mode=cs.CS_METRIC_SOFTMIN_S2))
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    for _ in range(3):  # interleaved on two streams: private scratch per graph
        ga.launch(s1)
        gb.launch(s2)
    ga.sync(s1)
    gb.sync(s2)
    ref_g = scene.query_grad(qa, 1.0, grad_out=up)
    ref_b = scene.query(qb, 0.5, params=cs.QueryParams(mode=cs.CS_METRIC_SOFTMIN_S2))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(ga.out["grad_centres"].cpu().numpy(), ref_g.cpu().numpy())
    _same(gb.out, ref_b, ["metric", "collide"])
    ga.close()
    gb.close()


def test_graph_rejects_host_io_and_bad_handles(cs, table):
    _, scene = table
    prims = torch.zeros((8, 4), device="cuda")
    prims[:, 3] = 0.1
    p = cs.QueryParams().to_c()
    p.host_io = 1
    import ctypes
    h = ctypes.c_void_p()
    out = torch.empty(8, device="cuda")
    st = cs.abi.cs_graph_create(scene.handle, 0, prims, 8, 1.0, out, None, None, None, p, h)
    assert st == cs.abi.CS_ERR_INVALID_ARG
    assert cs.abi.cs_graph_launch(ctypes.c_void_p(), None) == cs.abi.CS_ERR_BAD_HANDLE
    assert cs.abi.cs_graph_kernels(ctypes.c_void_p()) == -1


def test_autotune_records_a_listed_shape(cs, table):
    _, scene = table
    q = torch.as_tensor(S.arm_queries(configs=256), device="cuda")
    best, ms = scene.autotune(q, 1.0, reps=2)
    ids = cs.abi.cs_tile_configs()
    assert best in ids and set(ms) == set(ids)
    assert all(v > 0 for v in ms.values()) and ms[best] == min(ms.values())
    tuned = scene.query(q, 1.0, params=cs.QueryParams(tile_config=cs.abi.CS_TILE_TUNED), want_count=True)
    chosen = scene.query(q, 1.0, params=cs.QueryParams(tile_config=best), want_count=True)
    torch.cuda.synchronize()
    _same(tuned, chosen, ["metric", "collide", "count"])


def test_sweep_graph_replays_the_call(cs, table):
    """A captured conservatism sweep (cs_params.sweep_count) replays the
    call bit for bit, groups included."""
    _, scene = table
    sweep = (0.0, 0.5, 1.0, 2.0)
    d = torch.as_tensor(S.arm_queries(configs=625), device="cuda").contiguous()  # 40,000 spheres
    params = cs.QueryParams(group_size=64, sweep=sweep)
    g = cs.QueryGraph(scene, d, 0.0, params=params, want_count=True)
    out = g.launch()
    torch.cuda.synchronize()
    ref = scene.query(d, 0.0, params=params, want_count=True)
    torch.cuda.synchronize()
    for k in ("metric", "collide", "count", "group_metric", "group_collide"):
        np.testing.assert_array_equal(out[k].cpu().numpy().view(np.uint8), ref[k].cpu().numpy().view(np.uint8),
                                      err_msg=k)
    g.close()
