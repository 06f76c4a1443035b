"""cs_mppi_step (one fused MPPI iteration) against the FP64 MPPI oracle.

Inputs are dyadic (dt = 1/8, controls and perturbations on a 2^-10 grid), so
the FP32 rollout on the device is exact and both sides see the same sphere
centres.  Tolerances are derived from the oracle alone:
- per position, the metric tolerance of the parity contract (1e-5 relative,
  plus the Eq. 8 cancellation term), widened for positions with a pair in
  the cutoff band by the most that one membership flip can move a mean
  (mean + eps d_max per flipped pair over the remaining neighbours);
- per rollout, w_collision times the sum of those plus 4e-6 of the task and
  control sums (FP32 accumulation of T + 1 and T terms);
- weights: a common cost error bounded by D moves each weight by a factor
  within exp(+-2 D / lambda), plus 1e-6 for the FP32 exponential;
- the update: the weight error times |eps|, plus FP32 rounding of the sum.
"""
import numpy as np
import pytest

import cs_synth as S
import oracle
from oracle import mppi as omppi

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def cs(cuda_device):
    import paper_2609_35619_b300 as cs
    return cs


@pytest.fixture(scope="module")
def room(cs):
    sc = S.drone_scene(n=200_000)
    return sc, cs.Scene(sc["means"], sc["scales"], sc["quats"], sc["opacity"])


def _dyadic(a, bits=10):
    return (np.round(np.asarray(a, np.float64) * 2 ** bits) / 2 ** bits).astype(np.float32)


def _inputs(K, T, seed):
    rng = np.random.default_rng(seed)
    x0 = _dyadic([3.0, 2.5, 1.5])
    U = _dyadic(np.tile([0.4, -0.2, 0.05], (T, 1)) + rng.normal(0, 0.1, (T, 3)))
    eps = _dyadic(rng.normal(0, 0.6, (K, T, 3)))
    return x0, U, eps


def _tolerances(sc, d, res_pos, orc):
    p = oracle.Params()
    m = res_pos["mean_cost"]
    b = res_pos["band_cut"].astype(np.float64)
    n = res_pos["count_nbr"].astype(np.float64)
    strong = res_pos["cond"] > 50.0
    tol = 1e-5 * np.abs(m) + np.where(strong, 16 * U32 * p.gamma * res_pos["cond"] * np.abs(m), 0.0)
    tol += np.where(b > 0, (np.abs(m) + p.eps * p.d_max) * b / np.maximum(n - b, 1.0), 0.0)
    tol_col = tol.reshape(d.K, d.T).sum(1)
    tol_C = d.w_collision * tol_col + 4e-6 * (orc["task"] + orc["control"]) + 1e-7
    return tol_C


@pytest.mark.parametrize("K,T,ns,lam", [(256, 32, 1.0, 1.0), (1000, 16, 0.0, 0.3), (64, 32, 2.0, 5.0)])
def test_mppi_step_matches_oracle(cs, room, K, T, ns, lam):
    sc, scene = room
    x0, U, eps = _inputs(K, T, seed=K + T)
    d = omppi.MppiDesc(K=K, T=T, dt=0.125, radius=0.15, nsigma=ns, lam=lam, w_collision=10.0, w_goal=0.1,
                       w_terminal=1.0, w_control=0.01, goal=(4.5, 1.0, 1.25))
    out = cs.mppi_step(scene, x0, U, eps, dt=d.dt, radius=d.radius, nsigma=ns, lam=lam, w_collision=d.w_collision,
                       w_goal=d.w_goal, w_terminal=d.w_terminal, w_control=d.w_control, goal=d.goal)
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy().astype(np.float64) for k, v in out.items()}
    orc = omppi.step(sc, x0.astype(np.float64), U.astype(np.float64), eps.astype(np.float64), d)
    # the rollout positions are exact in FP32 (dyadic inputs): the oracle's
    # per-position metric gives the tolerance of each rollout's cost
    pos = orc["positions"].reshape(-1, 3)
    res_pos = oracle.query(sc, np.c_[pos, np.full(len(pos), d.radius)], 0, ns)
    tol_C = _tolerances(sc, d, res_pos, orc)
    err_C = np.abs(g["cost"] - orc["cost"])
    assert (err_C <= tol_C).all(), (err_C[err_C > tol_C][:4], tol_C[err_C > tol_C][:4])
    assert orc["collision"].max() > 0, "the rollouts should meet the scene"
    # rollout collision flags: exact unless a position has a pair in the collision band
    flags = res_pos["collide"].reshape(K, T).any(1)
    band = (res_pos["band_in"] > 0).reshape(K, T).any(1)
    np.testing.assert_array_equal(g["collide"][~band].astype(bool), flags[~band])
    # Eq. 10 weights
    D = tol_C.max()
    w = orc["weights"]
    tol_w = w * (np.expm1(2 * D / lam) + 1e-6) + 1e-9
    err_w = np.abs(g["weights"] - w)
    assert (err_w <= tol_w).all(), (err_w.max(), tol_w[err_w.argmax()])
    assert abs(g["weights"].sum() - 1) < 1e-5
    # update of the nominal sequence
    ae = np.abs(eps.astype(np.float64))
    tol_U = np.einsum("k,ktd->td", tol_w, ae) + 4 * K * U32 * np.einsum("k,ktd->td", w, ae) + 4 * U32 * np.abs(U)
    err_U = np.abs(g["U"] - orc["U"])
    assert (err_U <= tol_U + 1e-9).all(), (err_U.max(), tol_U.max())


def test_mppi_step_is_deterministic_and_updates_in_place(cs, room):
    sc, scene = room
    x0, U, eps = _inputs(512, 24, seed=3)
    a = cs.mppi_step(scene, x0, U, eps)
    b = cs.mppi_step(scene, x0, U, eps)
    torch.cuda.synchronize()
    for k in a:
        np.testing.assert_array_equal(a[k].cpu().numpy(), b[k].cpu().numpy(), err_msg=k)
    dU = torch.as_tensor(U, device="cuda").contiguous()
    c = cs.mppi_step(scene, x0, dU, eps, out={"U": dU, "cost": torch.empty(512, device="cuda"),
                                               "weights": torch.empty(512, device="cuda"),
                                               "collide": torch.empty(512, dtype=torch.uint8, device="cuda")})
    torch.cuda.synchronize()
    np.testing.assert_array_equal(c["U"].cpu().numpy(), a["U"].cpu().numpy())


def test_mppi_step_rejects_bad_arguments(cs, room):
    _, scene = room
    x0, U, eps = _inputs(8, 4, seed=4)
    with pytest.raises(cs.CsError):
        cs.mppi_step(scene, x0, U, eps, lam=0.0)
    with pytest.raises(cs.CsError):
        cs.mppi_step(scene, x0, U, eps, dt=-1.0)
    with pytest.raises(cs.CsError):
        cs.mppi_step(scene, x0, U, eps, w_goal=-1.0)


def test_mppi_graph_replays_the_iteration(cs, room):
    """The captured iteration equals cs_mppi_step bit for bit, and an
    in-place loop of captured iterations equals the same loop of calls."""
    _, scene = room
    x0, U, eps = _inputs(384, 20, seed=5)
    rng = np.random.default_rng(6)
    more = [_dyadic(rng.normal(0, 0.6, eps.shape)) for _ in range(3)]
    dx0 = torch.as_tensor(x0, device="cuda")
    dU = torch.as_tensor(U, device="cuda").contiguous()
    deps = torch.as_tensor(eps, device="cuda").contiguous()
    g = cs.MppiGraph(scene, dx0, dU, deps, in_place=True)
    assert g.kernels > 5
    U_ref = torch.as_tensor(U, device="cuda").contiguous()
    for it in range(3):
        deps.copy_(torch.as_tensor(more[it]))
        g.launch()
        ref = cs.mppi_step(scene, dx0, U_ref, torch.as_tensor(more[it], device="cuda"))
        U_ref = ref["U"].clone()
        g.sync()
        torch.cuda.synchronize()
        for k in ("U", "cost", "weights", "collide"):
            np.testing.assert_array_equal(g.out[k].cpu().numpy(), ref[k].cpu().numpy(), err_msg=f"{k} it {it}")
    g.close()
