"""Pins of the MPPI oracle (oracle/mppi.py) against values fixed by the
definitions of Section II-D, not by the oracle itself: closed-form rollouts,
a two-rollout example computed by hand, the limits of Eq. 10, and the
collision term against the closed form of one isotropic Gaussian."""
import math

import numpy as np

import oracle
from oracle import mppi


def _far_scene():
    # one Gaussian a kilometre away: no rollout here has a neighbour
    return {"means": np.array([[1e3, 1e3, 1e3]], np.float32), "scales": np.full((1, 3), 0.01, np.float32),
            "quats": np.array([[1, 0, 0, 0]], np.float32), "opacity": np.ones(1, np.float32)}


def test_rollout_constant_velocity_closed_form():
    x0 = np.array([0.5, -1.0, 2.0])
    U = np.tile([0.3, 0.2, -0.1], (7, 1))
    x, u = mppi.rollout(x0, U, np.zeros((3, 7, 3)), 0.25)
    for t in range(7):  # x[k, t] is the position after t + 1 steps
        np.testing.assert_allclose(x[:, t, :], np.tile(x0 + (t + 1) * 0.25 * U[0], (3, 1)), rtol=0, atol=1e-14)
    np.testing.assert_array_equal(u, np.tile(U, (3, 1, 1)))


def test_two_rollouts_by_hand():
    # K = 2, T = 2, dt = 0.5, x0 = 0, U = (1, 0, 0) twice, goal (1, 0, 0);
    # rollout 0 has no perturbation, rollout 1 adds (0, 1, 0) at both steps.
    # rollout 0: x = (0.5,0,0), (1,0,0); task = 1*(0.25 + 0) + 2*0 = 0.25;
    #            control = 0.5*(1 + 1) = 1;               C0 = 1.25
    # rollout 1: x = (0.5,0.5,0), (1,1,0); task = 1*(0.5 + 1) + 2*1 = 3.5;
    #            control = 0.5*(2 + 2) = 2;               C1 = 5.5
    # Eq. 10 with lambda = 1: w1 = e^-4.25 / (1 + e^-4.25), w0 = 1 - w1;
    # update: U' = U + w1 * (0, 1, 0) at both steps.
    d = mppi.MppiDesc(K=2, T=2, dt=0.5, radius=0.1, nsigma=1.0, lam=1.0, w_collision=10.0, w_goal=1.0,
                      w_terminal=2.0, w_control=0.5, goal=(1.0, 0.0, 0.0))
    U = np.array([[1.0, 0, 0], [1.0, 0, 0]])
    eps = np.zeros((2, 2, 3))
    eps[1, :, 1] = 1.0
    r = mppi.step(_far_scene(), np.zeros(3), U, eps, d)
    np.testing.assert_allclose(r["collision"], [0.0, 0.0], atol=0)
    np.testing.assert_allclose(r["task"], [0.25, 3.5], rtol=1e-15)
    np.testing.assert_allclose(r["control"], [1.0, 2.0], rtol=1e-15)
    np.testing.assert_allclose(r["cost"], [1.25, 5.5], rtol=1e-15)
    w1 = math.exp(-4.25) / (1 + math.exp(-4.25))
    np.testing.assert_allclose(r["weights"], [1 - w1, w1], rtol=1e-14)
    np.testing.assert_allclose(r["U"], [[1.0, w1, 0.0], [1.0, w1, 0.0]], rtol=1e-14, atol=1e-16)


def test_softmin_weights_limits_and_shift_invariance():
    rng = np.random.default_rng(0)
    C = rng.uniform(0, 10, 50)
    w = mppi.weights(C, 0.7)
    assert abs(w.sum() - 1) < 1e-14 and (w > 0).all()
    np.testing.assert_allclose(mppi.weights(C + 123.0, 0.7), w, rtol=1e-12)
    # lambda -> 0: all mass on the cheapest rollout; lambda -> inf: uniform
    cold = mppi.weights(C, 1e-4)
    assert cold.argmax() == C.argmin() and cold.max() > 1 - 1e-12
    np.testing.assert_allclose(mppi.weights(C, 1e12), np.full(50, 1 / 50), rtol=1e-9)
    # ratio of two weights is exp(-(C_a - C_b) / lambda)
    np.testing.assert_allclose(w[3] / w[7], math.exp(-(C[3] - C[7]) / 0.7), rtol=1e-12)


def test_equal_costs_move_nominal_by_mean_perturbation():
    rng = np.random.default_rng(1)
    K, T = 16, 5
    eps = rng.normal(size=(K, T, 3))
    # w_goal = w_terminal = w_control = 0 and a far scene: every cost is 0
    d = mppi.MppiDesc(K=K, T=T, w_goal=0.0, w_terminal=0.0, w_control=0.0)
    r = mppi.step(_far_scene(), np.zeros(3), np.zeros((T, 3)), eps, d)
    np.testing.assert_allclose(r["weights"], np.full(K, 1 / K), rtol=1e-14)
    np.testing.assert_allclose(r["U"], eps.mean(0), rtol=1e-12, atol=1e-15)


def test_collision_term_one_isotropic_gaussian_closed_form():
    # one isotropic Gaussian (std s) at the origin; a one-step rollout ends at
    # distance D; with a sphere of radius r the conservative distance is
    # st2 = max(0, D^2 - 2 n s D) / r^2 and the collision term is the Eq. 11
    # cost of that single neighbour, d_max exp(-gamma max(st2 - s_min, 0)).
    s, r, n, D = 0.05, 0.2, 1.5, 0.35
    scene = {"means": np.zeros((1, 3), np.float32), "scales": np.full((1, 3), s, np.float32),
             "quats": np.array([[1, 0, 0, 0]], np.float32), "opacity": np.ones(1, np.float32)}
    p = oracle.Params()
    st2 = max(0.0, D * D - 2 * n * s * D) / (r * r)
    want = p.d_max * math.exp(-p.gamma * max(st2 - p.s_min, 0.0))
    d = mppi.MppiDesc(K=1, T=1, dt=1.0, radius=r, nsigma=n, w_goal=0.0, w_terminal=0.0, w_control=0.0)
    U = np.array([[0.0, D, 0.0]], np.float32).astype(np.float64)
    r_ = mppi.step(scene, np.zeros(3), U, np.zeros((1, 1, 3)), d)
    # the FP32 inputs (scale, centre) are rounded before the oracle's FP64 work
    np.testing.assert_allclose(r_["collision"], [want], rtol=1e-6)
    np.testing.assert_allclose(r_["cost"], [d.w_collision * want], rtol=1e-6)
