"""cs_query_fwd_grad: the forward outputs and the adjoint of a sphere batch
from one fused launch.

- The gradient must have exactly the bits of cs_query_grad: the adjoint's
  arithmetic is unchanged, the forward reductions only ride along.
- The forward outputs are checked against the FP64 oracle with the parity
  contract's tolerances (the same check as cs_query).  They come from the
  adjoint's square root (u rsqrt(u)), so against cs_query they may differ in
  the last bits of the metric, and only for rows with a pair in a decision
  band in the count or flag.
- Group outputs, host buffers and the argument checks as for cs_query.
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


def _scene(cs, sc):
    return cs.Scene(sc["means"], sc["scales"], sc["quats"], sc.get("opacity"))


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("nsigma", [0.0, 1.0, 2.0])
def test_fused_matches_oracle_and_adjoint(cs, mode, nsigma):
    sc = S.tiny_scene()
    q = S.tiny_queries()
    scene = _scene(cs, sc)
    G = 7
    rng = np.random.default_rng(3)
    up = torch.as_tensor(rng.normal(size=(q.shape[0] + G - 1) // G).astype(np.float32), device="cuda")
    p = cs.QueryParams(mode=mode, group_size=G)
    fused = scene.query_fwd_grad(torch.as_tensor(q), nsigma, grad_out=up, params=p, want_count=True)
    grad = scene.query_grad(torch.as_tensor(q), nsigma, grad_out=up, params=p)
    fwd = scene.query(torch.as_tensor(q), nsigma, params=p, want_count=True)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(fused["grad"].cpu().numpy().view(np.uint32), grad.cpu().numpy().view(np.uint32))
    f = to_np({k: v for k, v in fused.items() if k != "grad"})
    orc = oracle.query(sc, q, 0, nsigma, oracle.Params())
    compare(f, orc, mode, oracle.Params(), f"fused mode={mode} nsigma={nsigma}")
    # against the forward call: the same flags and counts outside the decision bands
    a = to_np(fwd)
    ok = (orc["band_cut"] == 0) & (orc["band_in"] == 0)
    np.testing.assert_array_equal(f["count"][ok], a["count"][ok])
    np.testing.assert_array_equal(f["collide"][ok], a["collide"][ok])
    # the groups are the forward's group epilogue over the fused rows
    ng = f["group_metric"].shape[0]
    gm = np.array([f["metric"][i * G:(i + 1) * G].astype(np.float64).sum() for i in range(ng)])
    np.testing.assert_allclose(f["group_metric"], gm, rtol=1e-6)
    gc = np.array([f["collide"][i * G:(i + 1) * G].max() for i in range(ng)])
    np.testing.assert_array_equal(f["group_collide"], gc)


def test_fused_tabletop_pose_batch(cs):
    """The benchmark's pose spheres (full size) through the pose chain: the
    fused launch against the adjoint bit for bit, and sampled rows of the
    forward outputs against the oracle."""
    sc = S.tabletop_scene()
    scene = _scene(cs, sc)
    poses, offs, radius = S.trajectory_poses()
    dp = torch.as_tensor(poses, device="cuda")
    do = torch.as_tensor(offs, device="cuda")
    sph = cs.pose_spheres(dp, do, radius)
    K = offs.shape[0]
    p = cs.QueryParams(group_size=K)
    fused = scene.query_fwd_grad(sph, 1.0, params=p, want_count=True)
    grad = scene.query_grad(sph, 1.0, params=p)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(fused["grad"].cpu().numpy().view(np.uint32), grad.cpu().numpy().view(np.uint32))
    rows = np.random.default_rng(5).choice(sph.shape[0], 400, replace=False)
    s_np = sph.cpu().numpy()[rows]
    orc = oracle.query(sc, s_np, 0, 1.0, oracle.Params())
    f = {k: v.cpu().numpy()[rows] for k, v in fused.items() if k in ("metric", "collide", "count")}
    rep = compare(f, orc, 0, oracle.Params(), "fused pose batch")
    assert (orc["count_nbr"] > 0).mean() > 0.2, rep


def test_fused_host_io_and_arguments(cs):
    sc = S.tiny_scene()
    q = S.tiny_queries()[:300]
    scene = _scene(cs, sc)
    Q = q.shape[0]
    m = np.zeros(Q, np.float32)
    c = np.zeros(Q, np.uint8)
    g = np.zeros((Q, 3), np.float32)
    p = cs.QueryParams().to_c()
    p.host_io = 1
    cs.check(cs.abi.cs_query_fwd_grad(scene._h, cs.CS_PRIM_SPHERE, q, Q, 1.0, None, m, c, g, p))
    dev = scene.query_fwd_grad(torch.as_tensor(q), 1.0)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(m, dev["metric"].cpu().numpy())
    np.testing.assert_array_equal(c, dev["collide"].cpu().numpy())
    np.testing.assert_array_equal(g, dev["grad"].cpu().numpy())
    e = S.ellipsoid_queries(4, q[:, :3].astype(np.float64)).astype(np.float32)
    gg = torch.empty((e.shape[0], 3), device="cuda")
    with pytest.raises(cs.CsError):  # spheres only
        cs.check(cs.abi.cs_query_fwd_grad(scene._h, cs.CS_PRIM_ELLIPSOID, torch.as_tensor(e, device="cuda"),
                                          e.shape[0], 1.0, None, None, None, gg, None))
    for mode in (cs.CS_METRIC_MIN_S2, cs.CS_METRIC_SOFTMIN_S2, cs.CS_METRIC_FLAGS):
        with pytest.raises(cs.CsError):
            scene.query_fwd_grad(torch.as_tensor(q), 1.0, params=cs.QueryParams(mode=mode))
    with pytest.raises(cs.CsError):  # no sweep
        scene.query_fwd_grad(torch.as_tensor(q), 1.0, params=cs.QueryParams(sweep=(0.0, 1.0)))
