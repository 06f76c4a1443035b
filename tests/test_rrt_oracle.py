"""Pins of the RRT oracle (oracle/rrt.py) against values fixed by the steps
of the extension and by the closed form of Section II-B, not by the oracle
itself."""
import math

import numpy as np

import oracle
from oracle import rrt


def _far_scene():
    return {"means": np.array([[1e3, 1e3, 1e3]], np.float32), "scales": np.full((1, 3), 0.01, np.float32),
            "quats": np.array([[1, 0, 0, 0]], np.float32), "opacity": np.ones(1, np.float32)}


def test_nearest_breaks_ties_by_lowest_index():
    nodes = np.array([[1, 0, 0], [0, 1, 0], [-1, 0, 0], [0, 0, 2]], np.float32)
    # the origin is at distance 1 from nodes 0, 1, 2: node 0 wins
    near = rrt.nearest(nodes, 4, np.array([[0, 0, 0], [0, 0, 1.9], [-0.9, 0.1, 0]], np.float32))
    np.testing.assert_array_equal(near, [0, 3, 2])
    # only the first `count` nodes take part
    np.testing.assert_array_equal(rrt.nearest(nodes, 3, np.array([[0, 0, 1.9]], np.float32)), [0])


def test_steer_limits_the_edge_length():
    x = np.array([1.0, -2.0, 0.5], np.float32)
    far = np.array([4.0, 2.0, 0.5], np.float32)  # 5 m away along (3, 4, 0) / 5
    new = rrt.steer(x, far, 0.5)
    np.testing.assert_allclose(new, [1.3, -1.6, 0.5], rtol=0, atol=2e-6)
    assert abs(np.linalg.norm(new.astype(np.float64) - x) - 0.5) < 1e-6
    near = np.array([1.2, -2.1, 0.6], np.float32)
    np.testing.assert_array_equal(rrt.steer(x, near, 0.5), near)  # within reach: the sample itself


def test_edge_points_are_evenly_spaced_and_end_at_the_new_node():
    x = np.array([0.0, 0.0, 0.0], np.float32)
    new = np.array([0.8, -0.4, 0.2], np.float32)
    pts = rrt.edge_points(x, new, 8)
    np.testing.assert_array_equal(pts[-1], new)
    for m in range(8):
        np.testing.assert_allclose(pts[m], new.astype(np.float64) * (m + 1) / 8, rtol=0, atol=1e-7)


def test_edge_collision_at_the_closed_form_radius():
    # one isotropic Gaussian (std s) at the origin; the edge runs parallel to x
    # at distance D, with its midpoint (M even) at the closest approach: it
    # collides iff D < D* = n s + sqrt(n^2 s^2 + r^2) (Section II-B, Eq. 5-8)
    s, r, n = 0.05, 0.1, 1.0
    dstar = n * s + math.sqrt(n * n * s * s + r * r)
    scene = {"means": np.zeros((1, 3), np.float32), "scales": np.full((1, 3), s, np.float32),
             "quats": np.array([[1, 0, 0, 0]], np.float32), "opacity": np.ones(1, np.float32)}
    d = rrt.RrtDesc(B=2, M=8, step=10.0, radius=r, nsigma=n, capacity=16)
    for D, want in ((dstar * (1 - 1e-3), 1), (dstar * (1 + 1e-3), 0)):
        nodes = np.zeros((16, 3), np.float32)
        nodes[0] = (-0.4, D, 0.0)
        out = rrt.extend(scene, nodes, np.full(16, -1), 1,
                         np.array([[0.4, D, 0.0], [0.4, D, 0.0]], np.float32), d)
        np.testing.assert_array_equal(out["edge_collide"], [want, want])
        assert out["count"] == 1 + 2 * (1 - want)


def test_insertion_order_parents_and_capacity():
    d = rrt.RrtDesc(B=4, M=4, step=1.0, radius=0.1, capacity=4)
    nodes = np.zeros((4, 3), np.float32)
    nodes[1] = (5.0, 0.0, 0.0)
    samples = np.array([[0.1, 0, 0], [5.2, 0, 0], [0.0, 0.3, 0], [5.0, 0.4, 0]], np.float32)
    out = rrt.extend(_far_scene(), nodes, np.array([-1, 0, -1, -1]), 2, samples, d)
    np.testing.assert_array_equal(out["nearest"], [0, 1, 0, 1])
    assert (out["edge_collide"] == 0).all()
    assert out["count"] == 4  # capacity: the first two free edges only
    np.testing.assert_array_equal(out["nodes"][2:], samples[:2])
    np.testing.assert_array_equal(out["parent"][2:], [0, 1])
