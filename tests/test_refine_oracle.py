"""Pins of the path-refinement oracle (oracle/refine.py) against values
fixed outside it: B-spline identities (partition of unity, endpoint
interpolation, the curve of collinear evenly spaced control points is their
segment), the FP32 basis against the FP64 closed form, and the limits of the
Eq. 10 update."""
import numpy as np

import oracle
from oracle import refine as orf


def _empty_scene():
    return {"means": np.array([[1e3, 1e3, 1e3]], np.float32), "scales": np.full((1, 3), 0.01, np.float32),
            "quats": np.array([[1, 0, 0, 0]], np.float32), "opacity": np.ones(1, np.float32)}


def test_basis_partition_of_unity_and_float32_order():
    u = np.linspace(0, 1, 101)
    np.testing.assert_allclose(orf.basis(u).sum(-1), 1.0, rtol=0, atol=1e-15)
    for M in (1, 3, 8):
        for m in range(M):
            b32 = np.array(orf.basis32(m, M), np.float64)
            np.testing.assert_allclose(b32, orf.basis(m / M), rtol=0, atol=4e-7)


def test_spline_interpolates_endpoints_and_straight_polygon():
    rng = np.random.default_rng(1)
    P = rng.uniform(-1, 1, (7, 3)).astype(np.float32)
    pts = orf.points(P, 5)
    assert pts.shape == ((7 + 1) * 5 + 1, 3)
    np.testing.assert_allclose(pts[0], P[0], atol=1e-6)
    np.testing.assert_array_equal(pts[-1], P[-1])
    # collinear control points: every sample lies on the segment P0 -> P_{N-1}
    a, b = np.array([0.1, -0.2, 0.3]), np.array([1.1, 0.8, -0.7])
    L = (a[None] + np.linspace(0, 1, 6)[:, None] * (b - a)[None]).astype(np.float32)
    s = orf.points(L, 4).astype(np.float64)
    t = (s - a) @ (b - a) / np.dot(b - a, b - a)
    np.testing.assert_allclose(s, a[None] + t[:, None] * (b - a)[None], atol=2e-6)
    assert (np.diff(t) >= -1e-7).all() and abs(t[0]) < 1e-6 and abs(t[-1] - 1) < 1e-6


def test_uniform_weights_move_by_the_mean_perturbation():
    # no collision anywhere and lambda huge: Eq. 10 weights are uniform and
    # the interior control points move by the mean perturbation
    rng = np.random.default_rng(2)
    P = rng.uniform(-1, 1, (6, 3)).astype(np.float32)
    d = orf.RefineDesc(K=16, N=6, M=4, lam=1e12, w_length=1.0, w_collision=0.0)
    eps = rng.normal(0, 0.05, (16, 6, 3)).astype(np.float32)
    out = orf.refine(_empty_scene(), P, eps, d)
    np.testing.assert_allclose(out["weights"], 1 / 16, rtol=1e-9)
    mean = eps.astype(np.float64).mean(0)
    np.testing.assert_allclose(out["ctrl"][1:-1], P[1:-1].astype(np.float64) + mean[1:-1], rtol=0, atol=1e-9)
    np.testing.assert_array_equal(out["ctrl"][[0, -1]], P[[0, -1]].astype(np.float64))


def test_small_lambda_picks_the_shortest_path():
    # a zig-zag polygon; one rollout straightens it: with a small lambda the
    # update takes that rollout's perturbation
    P = np.array([[0, 0, 0], [0.3, 0.4, 0], [0.6, -0.4, 0], [1, 0, 0]], np.float32)
    eps = np.zeros((3, 4, 3), np.float32)
    eps[1, 1] = [0, -0.4, 0]
    eps[1, 2] = [0, 0.4, 0]
    eps[2, 1] = [0, 0.3, 0]
    d = orf.RefineDesc(K=3, N=4, M=8, lam=1e-4, w_length=1.0, w_collision=0.0)
    out = orf.refine(_empty_scene(), P, eps, d)
    assert np.argmax(out["weights"]) == 1 and out["weights"][1] > 0.999
    np.testing.assert_allclose(out["ctrl"][1:3, 1], [0, 0], atol=1e-3)
    np.testing.assert_allclose(out["length"][1], 1.0, rtol=1e-6)


def test_collision_term_counts_the_metric_of_every_point():
    # one isotropic Gaussian at the path's midpoint: the collision cost is the
    # sum of the per-point mean costs of the query oracle, nothing else
    sc = {"means": np.array([[0.5, 0, 0]], np.float32), "scales": np.full((1, 3), 0.02, np.float32),
          "quats": np.array([[1, 0, 0, 0]], np.float32), "opacity": np.ones(1, np.float32)}
    P = np.array([[0, 0, 0], [0.33, 0.01, 0], [0.66, -0.01, 0], [1, 0, 0]], np.float32)
    d = orf.RefineDesc(K=1, N=4, M=8, radius=0.05, w_length=0.0, w_collision=1.0)
    out = orf.refine(sc, P, np.zeros((1, 4, 3), np.float32), d)
    pts = orf.points(P, 8)
    ref = oracle.query(sc, np.c_[pts, np.full(len(pts), 0.05, np.float32)], 0, 1.0)["mean_cost"].sum()
    np.testing.assert_allclose(out["collision"][0], ref, rtol=1e-12)
    assert ref > 0
