"""cs_path_refine (zeroth-order path refinement, one MPPI step over the
B-spline control points of a plan) against the FP64 refinement oracle.

The sample points are computed by both sides in float32 with the same
rounded operations, so both query the same sphere centres.  Tolerances, from
the oracle alone (as for the MPPI iteration):
- per sample, the metric tolerance of the parity contract (1e-5 relative
  plus the Eq. 8 cancellation term), widened where a pair sits in the cutoff
  band by the most one membership flip can move the mean;
- per rollout, w_collision times their sum plus w_length times the FP32
  accumulation bound of the polyline length ((P + 4) u times the sum of the
  segment lengths);
- weights: a cost error bounded by D moves each weight by a factor within
  exp(+-2 D / lambda), plus 1e-6 for the FP32 exponential;
- the update: the weight error times |eps|, plus FP32 rounding of the sum;
  the endpoints must not move at all.
"""
import numpy as np
import pytest

import cs_synth as S
import oracle
from oracle import refine as orf

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


def _plan(N, seed):
    rng = np.random.default_rng(seed)
    a, b = np.array([0.8, 0.7, 1.2]), np.array([5.2, 4.3, 1.6])
    t = np.linspace(0, 1, N)[:, None]
    P = a + t * (b - a) + np.r_[np.zeros((1, 3)), rng.normal(0, 0.25, (N - 2, 3)), np.zeros((1, 3))]
    return P.astype(np.float32)


def _tolerance_C(sc, d, orc):
    p = oracle.Params()
    res = orc["query"]  # the oracle's own per-sample metric
    m = res["mean_cost"]
    b = res["band_cut"].astype(np.float64)
    n = res["count_nbr"].astype(np.float64)
    strong = res["cond"] > 50.0
    tol = 1e-5 * np.abs(m) + np.where(strong, 16 * U32 * p.gamma * res["cond"] * np.abs(m), 0.0)
    tol += np.where(b > 0, (np.abs(m) + p.eps * p.d_max) * b / np.maximum(n - b, 1.0), 0.0)
    P = orc["points"].shape[1]
    return d.w_collision * tol.reshape(d.K, P).sum(1) + d.w_length * (P + 4) * U32 * orc["length"] + 1e-7


@pytest.mark.parametrize("K,N,M,ns,lam", [(128, 12, 6, 1.0, 1.0), (512, 6, 4, 0.0, 0.3), (48, 20, 4, 2.0, 3.0)])
def test_refine_step_matches_oracle(cs, room, K, N, M, ns, lam):
    sc, scene = room
    P = _plan(N, seed=N)
    eps = np.random.default_rng(K + N).normal(0, 0.12, (K, N, 3)).astype(np.float32)
    d = orf.RefineDesc(K=K, N=N, M=M, radius=0.1, nsigma=ns, lam=lam, w_length=1.0, w_collision=5.0)
    out = cs.path_refine(scene, P, eps, M=M, radius=d.radius, nsigma=ns, lam=lam, w_length=d.w_length,
                         w_collision=d.w_collision)
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy().astype(np.float64) for k, v in out.items()}
    orc = orf.refine(sc, P, eps, d)
    assert orc["collision"].max() > 0, "the perturbed paths should meet the scene"
    tol_C = _tolerance_C(sc, d, orc)
    err_C = np.abs(g["cost"] - orc["cost"])
    assert (err_C <= tol_C).all(), (err_C[err_C > tol_C][:4], tol_C[err_C > tol_C][:4])
    D = tol_C.max()
    w = orc["weights"]
    tol_w = w * (np.expm1(2 * D / lam) + 1e-6) + 1e-9
    err_w = np.abs(g["weights"] - w)
    assert (err_w <= tol_w).all(), (err_w.max(), tol_w[err_w.argmax()])
    ae = np.abs(eps.astype(np.float64))
    ae[:, [0, -1]] = 0.0
    tol_P = np.einsum("k,knd->nd", tol_w, ae) + 4 * K * U32 * np.einsum("k,knd->nd", w, ae) + 4 * U32 * np.abs(P)
    err_P = np.abs(g["ctrl"] - orc["ctrl"])
    assert (err_P <= tol_P + 1e-9).all(), (err_P.max(), tol_P.max())
    np.testing.assert_array_equal(g["ctrl"][[0, -1]], P[[0, -1]].astype(np.float64))


def test_refine_shortens_a_free_zigzag(cs, room):
    """Far from the scene, many rollouts and a small lambda: the step moves the
    interior control points so the path gets shorter (the oracle agrees)."""
    sc, scene = room
    P = np.array([[10, 10, 10], [10.3, 10.4, 10], [10.6, 9.6, 10], [11, 10, 10]], np.float32)
    eps = np.random.default_rng(1).normal(0, 0.2, (2048, 4, 3)).astype(np.float32)
    out = cs.path_refine(scene, P, eps, M=8, lam=0.01, w_collision=0.0)
    torch.cuda.synchronize()
    new = out["ctrl"].cpu().numpy()
    L = lambda c: np.linalg.norm(np.diff(orf.points(c, 8).astype(np.float64), axis=0), axis=1).sum()
    assert L(new) < 0.9 * L(P)


def test_refine_rejects_bad_arguments(cs, room):
    _, scene = room
    P = _plan(6, 1)
    eps = np.zeros((4, 6, 3), np.float32)
    with pytest.raises(cs.CsError):
        cs.path_refine(scene, P, eps, lam=0.0)
    with pytest.raises(cs.CsError):
        cs.path_refine(scene, P[:1], eps[:, :1], M=4)
    with pytest.raises(cs.CsError):
        cs.path_refine(scene, P, eps, M=0)
