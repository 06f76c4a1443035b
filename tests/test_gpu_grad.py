"""Adjoint kernel (cs_query_grad) and pose chain vs the FP64 oracle's
analytic gradient and central finite differences.

Tolerance: |g_gpu - g_oracle| <= (1e-4 + w) |g_oracle| + 1e-5 * scale, where
scale is the sum of the sizes of the terms the gradient sums (the oracle
returns it; parts that cancel count at their own size), and w bounds the
relative error of the weights the terms carry: Eq. 8 cancels, so FP32 st^2
carries an absolute error up to 8 u cond (cond = s^2 + n sqrt(sigma^2),
u = 2^-24), which the Eq. 11 weights exp(-gamma st^2) amplify by gamma and
the softmin weights exp(-st^2/tau) by 1/tau.  Rows with a pair within 1e-5 of
a kink of the gradient (st^2 = s_min, the Eq. 8 clamp, the cutoff) are
excluded and counted.
"""
import numpy as np
import pytest

import cs_synth as S
import oracle
from oracle import pose as opose

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cs(cuda_device):
    import paper_2609_35619_b300 as cs
    return cs


def _scene(cs, sc):
    return cs.Scene(sc["means"], sc["scales"], sc["quats"], sc["opacity"])


U32 = 2.0 ** -24


def _weight_rel(mode, cond, params=oracle.Params()):
    if mode in (0, 1):
        return 16 * U32 * params.gamma * cond
    if mode == 3:
        return 16 * U32 * cond / params.tau
    return 0.0 * cond


def _check(g_gpu, g_orc, scale, exclude, label, wrel=None):
    ok = ~exclude
    err = np.linalg.norm(g_gpu[ok] - g_orc[ok], axis=1)
    w = 0.0 if wrel is None else wrel[ok]
    tol = (1e-4 + w) * np.linalg.norm(g_orc[ok], axis=1) + 1e-5 * scale[ok] + 1e-12
    bad = err > tol
    assert not bad.any(), (f"{label}: {bad.sum()}/{ok.sum()} gradient mismatches; "
                           f"gpu={g_gpu[ok][bad][:3]} oracle={g_orc[ok][bad][:3]}")
    return int(exclude.sum())


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
@pytest.mark.parametrize("prim_type", [0, 1])
def test_adjoint_matches_oracle(cs, mode, prim_type):
    sc = S.tiny_scene(n=3000)
    rng = np.random.default_rng(100 + mode)
    Q = 700
    c = rng.uniform(0, 2, (Q, 3))
    prims = (np.c_[c, rng.uniform(0.05, 0.25, Q)] if prim_type == 0
             else S.ellipsoid_queries(7, c)).astype(np.float32)
    scene = _scene(cs, sc)
    up = rng.normal(size=Q).astype(np.float32)
    for ns in (0.0, 1.0, 2.0):
        g = scene.query_grad(torch.as_tensor(prims), ns, grad_out=torch.as_tensor(up), prim_type=prim_type,
                             params=cs.QueryParams(mode=mode)).cpu().numpy()
        go, scale = oracle.grad(sc, prims, prim_type, ns, mode, grad_out=up.astype(np.float64),
                                return_scale=True)
        orc = oracle.query(sc, prims, prim_type, ns)
        excl = (orc["band_cut"] > 0) | (orc["band_kink"] > 0)
        _check(g, go, scale, excl, f"mode={mode} prim={prim_type} ns={ns}",
               wrel=_weight_rel(mode, orc["cond"]))


@pytest.mark.parametrize("mode,prim_type", [(0, 0), (3, 1), (2, 0)])
def test_adjoint_tile_shapes_give_the_same_bits(cs, mode, prim_type):
    """Every adjoint tile shape sums each lane's Gaussians in chunk order, so
    all shapes return the same bits; the default also matches the oracle."""
    sc = S.tiny_scene(n=3000)
    rng = np.random.default_rng(9)
    Q = 1500
    c = rng.uniform(0, 2, (Q, 3))
    prims = (np.c_[c, rng.uniform(0.05, 0.25, Q)] if prim_type == 0
             else S.ellipsoid_queries(9, c)).astype(np.float32)
    scene = _scene(cs, sc)
    up = torch.as_tensor(rng.normal(size=Q).astype(np.float32))
    outs = [scene.query_grad(torch.as_tensor(prims), 1.0, grad_out=up, prim_type=prim_type,
                             params=cs.QueryParams(mode=mode, tile_config=t)).cpu().numpy() for t in (1, 2, 3, 4)]
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])
    go, scale = oracle.grad(sc, prims, prim_type, 1.0, mode, grad_out=up.numpy().astype(np.float64),
                            return_scale=True)
    orc = oracle.query(sc, prims, prim_type, 1.0)
    _check(outs[1], go, scale, (orc["band_cut"] > 0) | (orc["band_kink"] > 0), f"shapes mode={mode}",
           wrel=_weight_rel(mode, orc["cond"]))


def test_adjoint_group_upstream(cs):
    sc = S.tiny_scene()
    q = S.tiny_queries(q=640)
    scene = _scene(cs, sc)
    G = 64
    up = np.random.default_rng(1).normal(size=q.shape[0] // G).astype(np.float32)
    g = scene.query_grad(torch.as_tensor(q), 1.0, grad_out=torch.as_tensor(up),
                         params=cs.QueryParams(group_size=G)).cpu().numpy()
    go, scale = oracle.grad(sc, q, 0, 1.0, grad_out=np.repeat(up, G).astype(np.float64), return_scale=True)
    orc = oracle.query(sc, q, 0, 1.0)
    _check(g, go, scale, (orc["band_cut"] > 0) | (orc["band_kink"] > 0), "group upstream",
           wrel=_weight_rel(0, orc["cond"]))


def test_adjoint_against_central_differences(cs):
    """Central differences (h = 1e-4 m) of the GPU metric itself agree with
    the GPU adjoint on rows where the metric is smooth across the stencil
    (rows where the oracle's own central differences match its analytic
    gradient; elsewhere a kink of Eq. 8/11 or of the neighbour set lies
    within h)."""
    sc = S.tiny_scene()
    rng = np.random.default_rng(2)
    Q = 200
    q = np.c_[rng.uniform(0.2, 1.8, (Q, 3)), rng.uniform(0.1, 0.25, Q)].astype(np.float32)
    scene = _scene(cs, sc)
    g = scene.query_grad(torch.as_tensor(q), 1.0, params=cs.QueryParams(mode=1)).cpu().numpy()
    h = 1e-4
    fd = np.zeros((Q, 3))
    fd_o = np.zeros((Q, 3))
    base = scene.query(torch.as_tensor(q), 1.0, params=cs.QueryParams(mode=1))
    for a in range(3):
        qp = q.astype(np.float64).copy()
        qm = q.astype(np.float64).copy()
        qp[:, a] += h
        qm[:, a] -= h
        qp, qm = qp.astype(np.float32), qm.astype(np.float32)
        step = qp[:, a].astype(np.float64) - qm[:, a].astype(np.float64)
        mp = scene.query(torch.as_tensor(qp), 1.0, params=cs.QueryParams(mode=1))["metric"]
        mm = scene.query(torch.as_tensor(qm), 1.0, params=cs.QueryParams(mode=1))["metric"]
        fd[:, a] = (mp.cpu().numpy().astype(np.float64) - mm.cpu().numpy().astype(np.float64)) / step
        fd_o[:, a] = (oracle.query(sc, qp, 0, 1.0)["sum_cost"] - oracle.query(sc, qm, 0, 1.0)["sum_cost"]) / step
    go = oracle.grad(sc, q, 0, 1.0, oracle.MODE_SUM)
    smooth = np.linalg.norm(fd_o - go, axis=1) <= 1e-3 * np.linalg.norm(go, axis=1) + 1e-9
    m = base["metric"].cpu().numpy().astype(np.float64)
    err = np.linalg.norm(g - fd, axis=1)[smooth]
    # FP32 metric differences over 2h: noise ~ 1e-6 |m| / h
    tol = 2e-3 * np.linalg.norm(g, axis=1)[smooth] + 1e-6 * np.abs(m[smooth]) / h + 1e-6
    assert (err <= tol).all(), (err[err > tol][:5], tol[err > tol][:5])
    assert smooth.sum() > Q // 2


def test_pose_chain_forward_and_adjoint(cs):
    poses, offs, r = S.trajectory_poses(trajectories=16, waypoints=16)
    P = poses.shape[0]
    tp = torch.as_tensor(poses, device="cuda")
    to = torch.as_tensor(offs, device="cuda")
    sph = cs.pose_spheres(tp, to, r).cpu().numpy()
    want = opose.centres(poses, offs).reshape(-1, 3)
    # the FP32 chain's derived bound (see test_collision_cost_autograd)
    delta = (16 * U32 * (np.linalg.norm(poses[:, :3], axis=1)[:, None] +
                         2 * np.linalg.norm(offs, axis=1)[None, :])).reshape(-1)
    assert (np.linalg.norm(sph[:, :3] - want, axis=1) <= delta).all()
    assert (sph[:, 3] == np.float32(r)).all()
    gc = np.random.default_rng(3).normal(size=(P * offs.shape[0], 3)).astype(np.float32)
    gp = cs.pose_spheres_grad(tp, to, torch.as_tensor(gc, device="cuda")).cpu().numpy()
    want_g = opose.pose_grad(poses, offs, gc.reshape(P, -1, 3))
    np.testing.assert_allclose(gp, want_g, rtol=1e-4, atol=1e-5)


def test_collision_cost_autograd(cs):
    """torch.autograd through CollisionCost (config 4: poses -> FP32 sphere
    centres -> metric summed over the K body spheres -> adjoint -> pose
    gradient) against the FP64 chain: oracle centres c* from the FP64 pose
    chain, the oracle metric and its analytic gradient there, pushed through
    the FP64 pose adjoint.  Section II-D sums the cost over the links.

    Derived tolerance.  The FP32 pose chain (R from sincosf/sinf, documented
    to 2 ulp, then c = t + R p, about a dozen roundings on each path) puts
    each centre within delta = 16 u (|t| + 2 |p_k|) of c* (u = 2^-24; the
    pose-chain test pins the same bound).  Over that ball the oracle gives:
      L_k = max(|g*(c*)|, max_i |g*(c* +- delta e_i)|)   the metric's slope,
      V_k = max_i |g*(c* +- delta e_i) - g*(c*)|          the gradient's change.
    Cost of a pose: the FP32 group sum of its K row metrics, so
      |cost - sum_k m*_k| <= sum_k (tol_k + sqrt(3) L_k delta_k) + gamma_m sum_k |m_k|,
    tol_k the row bound of the parity contract (1e-5 relative, widened only
    for cancelling rows), gamma_m the rounding of the K-term warp sum.
    Pose gradient: grad_t = sum_k g_k and grad_w = J^T sum_k (R p_k) x g_k with
    |J| <= 1, so with e_k = (1e-4 + w_k) |g*_k| + 1e-5 scale_k + sqrt(3) V_k,
      |grad_t - grad_t*| <= sum_k e_k + 32 u sum_k |g_k|,
      |grad_w - grad_w*| <= sum_k |p_k| (e_k + 32 u |g_k|).
    Poses with a row in the cutoff band or near a kink of the gradient (where
    neither the row nor its slope is single-valued) are left out and counted."""
    sc = S.tabletop_scene(n=200_000)
    poses, offs, r = S.trajectory_poses(trajectories=32, waypoints=16)
    scene = _scene(cs, sc)
    tp = torch.tensor(poses, device="cuda", requires_grad=True)
    to = torch.as_tensor(offs, device="cuda")
    cost = cs.CollisionCost.apply(tp, scene, to, r, 1.0, None)
    w = torch.as_tensor(np.random.default_rng(4).normal(size=poses.shape[0]).astype(np.float32), device="cuda")
    (cost * w).sum().backward()
    g = tp.grad.cpu().numpy()
    P, K = poses.shape[0], offs.shape[0]
    sph = opose.centres(poses, offs).reshape(-1, 3)                    # c*, FP64
    prims = np.c_[sph, np.full(sph.shape[0], r)].astype(np.float32)
    delta = (16 * U32 * (np.linalg.norm(poses[:, :3], axis=1)[:, None] +
                         2 * np.linalg.norm(offs, axis=1)[None, :])).reshape(-1)
    P_ = oracle.Params()
    orc = oracle.query(sc, prims, 0, 1.0, P_)
    wk = np.repeat(w.cpu().numpy(), K).astype(np.float64)
    g0, scale = oracle.grad(sc, prims, 0, 1.0, grad_out=wk, return_scale=True)
    shifted = []
    for ax in range(3):
        for sgn in (-1.0, 1.0):
            q = prims.copy().astype(np.float64)
            q[:, ax] += sgn * delta
            shifted.append(oracle.grad(sc, q.astype(np.float32), 0, 1.0, grad_out=wk))
    gn = np.stack([np.linalg.norm(x, axis=1) for x in shifted])
    unit = np.linalg.norm(oracle.grad(sc, prims, 0, 1.0), axis=1)       # the metric's own slope
    unit_sh = np.max([np.linalg.norm(oracle.grad(sc, np.c_[prims[:, :3] + sgn * delta[:, None] * np.eye(3)[ax],
                                                           prims[:, 3]].astype(np.float32), 0, 1.0), axis=1)
                      for ax in range(3) for sgn in (-1.0, 1.0)], axis=0)
    L = np.maximum(unit, unit_sh)
    V = np.max(np.stack([np.linalg.norm(x - g0, axis=1) for x in shifted]), axis=0)
    bad_rows = (orc["band_cut"] > 0) | (orc["band_kink"] > 0)
    ok = ~bad_rows.reshape(P, K).any(1)
    assert ok.sum() > 0.5 * P, f"only {ok.sum()} of {P} poses checked"
    # cost of each pose: the row bound of the parity contract (1e-5 relative,
    # widened by 16 u gamma cond_cost for rows whose Eq. 8 cancels strongly)
    from _parity import COND_STRICT, REL, summation_depth
    rows_m = orc["mean_cost"]
    strong = orc["cond_cost"] > COND_STRICT
    tol_row = (REL + np.where(strong, 16 * U32 * P_.gamma * orc["cond_cost"], 0.0)) * np.abs(rows_m)
    m = summation_depth(K, K)
    gam = m * U32 / (1 - m * U32)
    c_gpu = cost.detach().cpu().numpy().astype(np.float64)
    c_orc = rows_m.reshape(P, K).sum(1)
    c_tol = (tol_row + np.sqrt(3) * L * delta).reshape(P, K).sum(1) + gam * np.abs(rows_m).reshape(P, K).sum(1) + 1e-30
    c_err = np.abs(c_gpu - c_orc)
    assert (c_err[ok] <= c_tol[ok]).all(), (c_err[ok][c_err[ok] > c_tol[ok]][:5], c_tol[ok][c_err[ok] > c_tol[ok]][:5])
    # pose gradient
    want = opose.pose_grad(poses, offs, g0.reshape(P, K, 3))
    wrel = _weight_rel(0, orc["cond"])
    e = (1e-4 + wrel) * np.linalg.norm(g0, axis=1) + 1e-5 * scale + np.sqrt(3) * V
    gsz = np.linalg.norm(g0, axis=1)
    pk = np.tile(np.linalg.norm(offs, axis=1), P)
    tol_t = (e + 32 * U32 * gsz).reshape(P, K).sum(1)
    tol_w = (pk * (e + 32 * U32 * gsz)).reshape(P, K).sum(1)
    err_t = np.linalg.norm(g[:, :3] - want[:, :3], axis=1)
    err_w = np.linalg.norm(g[:, 3:] - want[:, 3:], axis=1)
    assert (err_t[ok] <= tol_t[ok] + 1e-12).all(), (err_t[ok][err_t[ok] > tol_t[ok]][:5], tol_t[ok][err_t[ok] > tol_t[ok]][:5])
    assert (err_w[ok] <= tol_w[ok] + 1e-12).all(), (err_w[ok][err_w[ok] > tol_w[ok]][:5], tol_w[ok][err_w[ok] > tol_w[ok]][:5])
    assert np.abs(want).max() > 0 and (np.abs(c_orc[ok]) > 0).sum() > 10
