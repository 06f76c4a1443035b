"""Pins of the oracle's diagnostic outputs, which the parity tests use to
exclude rows and to widen tolerances:

  cond       max over N_j of s^2 + n sqrt(sigma^2): the size of the two terms
             that Eq. 8 subtracts (its condition number times st^2)
  min_cond   s^2 + n sqrt(sigma^2) of the pair giving min st^2
  band_cut   pairs with |st^2 - S_cut| <= band S_cut (neighbour membership can
             flip in FP32), S_cut = s_min + ln(1/eps)/gamma
  band_in    pairs with |st^2 - 1| <= band (the Section II-E flag can flip)
  band_kink  pairs near a kink of the gradient: |st^2 - s_min| <= band
             max(1, |s_min|) (Eq. 11's max(., 0)), or the Eq. 8 clamp within
             band of switching, |raw| <= band (s^2 + n sqrt(sigma^2))
  cond_cost  cond over the pairs of N_j with st^2 >= s_min - band cond (Eq. 11 is
             flat below s_min, so cancellation there cannot reach the cost)
  gscale     |upstream| times the sum, over the terms of the gradient, of the
             norms of the two parts of d st^2/dc (-2 A d and the n sqrt(sigma^2)
             part), weighted as the metric weights the terms

Every expected value below is derived by hand from Eq. 5, 7, 8 and 11 with
inputs that are exact in binary (so the FP64 oracle reproduces them to the
last few ulps).  For a sphere of radius r and an isotropic Gaussian of
standard deviation s at distance D along x:
  s^2 = D^2/r^2,  sigma^2 = 4 s^2 D^2 / r^4,  sqrt(sigma^2) = 2 s D / r^2,
  st^2 = max(0, s^2 - n sqrt(sigma^2)),
  d st^2/dc = (-2 d + 2 n Sigma d / sqrt(d^T Sigma d)) / r^2 with the two
  parts of norms 2 D / r^2 and 2 n s / r^2.
"""
import math

import numpy as np
import pytest

import oracle


def _scene(means, stds, opacity=None):
    """Isotropic Gaussians (std per Gaussian) at the given means."""
    means = np.asarray(means, np.float32).reshape(-1, 3)
    n = means.shape[0]
    stds = np.broadcast_to(np.asarray(stds, np.float32), (n,))
    scales = np.repeat(stds[:, None], 3, 1).astype(np.float32)
    quats = np.tile(np.float32([1, 0, 0, 0]), (n, 1))
    op = np.ones(n, np.float32) if opacity is None else np.asarray(opacity, np.float32)
    return {"means": means, "scales": scales, "quats": quats, "opacity": op}


SPHERE_HALF = np.float32([[0, 0, 0, 0.5]])
SPHERE_ONE = np.float32([[0, 0, 0, 1.0]])


# ----------------------------------------------------------- cond, min_cond
def test_cond_and_min_cond_by_hand():
    """r = 0.5, n = 1.
    G_a: s = 1/4 at (0, 3/4, 0): s^2 = 9/4, sqrt(sigma^2) = 2 (1/4)(3/4)/(1/4) = 3/2,
         st^2 = 3/4, cond_a = 9/4 + 3/2 = 15/4.
    G_b: s = 1/8 at (1/2, 0, 0): s^2 = 1, sqrt(sigma^2) = 2 (1/8)(1/2)/(1/4) = 1/2,
         st^2 = 1/2, cond_b = 3/2.
    G_c: s = 1/4 at (3, 0, 0): s^2 = 36, sqrt(sigma^2) = 6, st^2 = 30 > S_cut:
         outside N_j, so its cond (42) must not count.
    cond = max(15/4, 3/2) = 15/4; min_cond = cond of the argmin pair (G_b,
    evaluated after G_a) = 3/2."""
    sc = _scene([[0, 0.75, 0], [0.5, 0, 0], [3, 0, 0]], [0.25, 0.125, 0.25])
    o = oracle.query(sc, SPHERE_HALF, 0, 1.0)
    assert o["count_nbr"][0] == 2
    assert o["cond"][0] == pytest.approx(15 / 4, rel=1e-14)
    assert o["min_cond"][0] == pytest.approx(3 / 2, rel=1e-14)
    assert o["min_s2"][0] == pytest.approx(0.5, rel=1e-14)
    # the square root matters: with n = 2, cond_a = 9/4 + 3 = 21/4 and cond_b = 1 + 1 = 2
    o2 = oracle.query(sc, SPHERE_HALF, 0, 2.0)
    assert o2["cond"][0] == pytest.approx(21 / 4, rel=1e-14)
    # st^2_a = max(0, 9/4 - 3) = 0, st^2_b = max(0, 1 - 1) = 0: G_a is the first minimum
    assert o2["min_s2"][0] == 0.0
    assert o2["min_cond"][0] == pytest.approx(21 / 4, rel=1e-14)
    # n = 0: cond = s^2 of the farthest neighbour; here s^2_a = 9/4, s^2_b = 1
    o0 = oracle.query(sc, SPHERE_HALF, 0, 0.0)
    assert o0["cond"][0] == pytest.approx(9 / 4, rel=1e-14)
    assert o0["min_cond"][0] == pytest.approx(1.0, rel=1e-14)


def test_cond_empty_set_is_zero():
    sc = _scene([[5, 5, 5]], [0.01])
    o = oracle.query(sc, SPHERE_HALF, 0, 1.0)
    assert o["count_nbr"][0] == 0 and o["cond"][0] == 0.0 and o["min_cond"][0] == 0.0


def test_cond_ellipsoid_scaling():
    """An ellipsoid with semi-axes (1/2, 1, 1) (no rotation) and a point
    Gaussian (s = 0) at (1/2, 0, 0): s^2 = (1/2)^2 / (1/2)^2 = 1, sigma^2 = 0,
    cond = 1; an isotropic s = 1/4 at (0, 1, 0): A d = (0, 1, 0), s^2 = 1,
    sqrt(sigma^2) = 2 sqrt(w^T Sigma w) = 2 (1/4) = 1/2, so at n = 2
    cond = 1 + 1 = 2 and st^2 = 0."""
    ell = np.float32([[0, 0, 0, 1, 0, 0, 0, 0.5, 1, 1]])
    o = oracle.query(_scene([[0.5, 0, 0]], [0.0]), ell, 1, 2.0)
    assert o["cond"][0] == pytest.approx(1.0, rel=1e-14)
    o = oracle.query(_scene([[0, 1, 0]], [0.25]), ell, 1, 2.0)
    assert o["cond"][0] == pytest.approx(2.0, rel=1e-14)
    assert o["min_s2"][0] == 0.0


# ------------------------------------------------------- band_cut, band_in
def _points_at_st2(values):
    """Point Gaussians (s = 0) on the x axis with st^2 = D^2 = value against
    the unit sphere at n = 0 (D rounded to float32: relative error of st^2
    below 1.2e-7, far inside the margins used)."""
    return _scene([[math.sqrt(v), 0, 0] for v in values], [0.0])


def test_band_cut_by_hand():
    p = oracle.Params()
    S = p.s_cut  # 1 + ln(1e6)/5
    assert S == pytest.approx(1 + 6 * math.log(10) / 5, rel=1e-15)
    vals = [S * (1 + 0.5e-5), S * (1 - 0.5e-5), S * (1 + 2e-5), S * (1 - 2e-5), 2.0]
    o = oracle.query(_points_at_st2(vals), SPHERE_ONE, 0, 0.0)
    assert o["band_cut"][0] == 2          # the two within 1e-5 relative of S_cut
    assert o["count_nbr"][0] == 3         # S(1 - 0.5e-5), S(1 - 2e-5) and 2
    o = oracle.query(_points_at_st2(vals), SPHERE_ONE, 0, 0.0, oracle.Params(band=1e-4))
    assert o["band_cut"][0] == 4          # the band scales with its parameter
    # the band is relative to S_cut: at gamma = 50, S_cut = 1.2763 and the
    # band is 1.276e-5 wide, so S_cut + 1.2e-5 lies in it and S_cut + 1.5e-5
    # does not
    p50 = oracle.Params(gamma=50.0)
    S50 = p50.s_cut
    o = oracle.query(_points_at_st2([S50 + 1.2e-5, S50 + 1.5e-5]), SPHERE_ONE, 0, 0.0, p50)
    assert o["band_cut"][0] == 1


def test_band_in_by_hand():
    vals = [1 + 0.5e-5, 1 - 0.5e-5, 1 + 2e-5, 1 - 2e-5, 0.25]
    o = oracle.query(_points_at_st2(vals), SPHERE_ONE, 0, 0.0)
    assert o["band_in"][0] == 2           # absolute band 1e-5 around 1
    assert o["count_in"][0] == 3          # 1 - 0.5e-5, 1 - 2e-5, 0.25
    o = oracle.query(_points_at_st2(vals), SPHERE_ONE, 0, 0.0, oracle.Params(band=3e-5))
    assert o["band_in"][0] == 4


# ---------------------------------------------------------------- band_kink
def test_band_kink_at_s_min_by_hand():
    """s_min = 2 (S_cut = 2 + ln(1e6)/5) separates the Eq. 11 kink from the
    collision threshold at 1: points at st^2 = 2 (1 +- 0.5e-5) are kinks,
    points at 2 (1 +- 4e-5) and at 1 are not."""
    p = oracle.Params(s_min=2.0)
    vals = [2 * (1 + 0.5e-5), 2 * (1 - 0.5e-5), 2 * (1 + 4e-5), 2 * (1 - 4e-5), 1.0]
    o = oracle.query(_points_at_st2(vals), SPHERE_ONE, 0, 0.0, p)
    assert o["band_kink"][0] == 2
    assert o["band_in"][0] == 1
    # |s_min| < 1: the band is absolute (band * max(1, |s_min|))
    p = oracle.Params(s_min=0.5)
    o = oracle.query(_points_at_st2([0.5 + 0.8e-5, 0.5 + 1.5e-5]), SPHERE_ONE, 0, 0.0, p)
    assert o["band_kink"][0] == 1


def test_band_kink_at_the_eq8_clamp_by_hand():
    """r = 1, n = 1, isotropic s = 1/4: raw = D^2 - 2 s D = D (D - 1/2) is zero
    at D = 1/2 (exactly, in binary), a kink of Eq. 8's max(., 0); at D = 3/4,
    raw = 3/16, far from 0 (and from s_min = 1)."""
    o = oracle.query(_scene([[0.5, 0, 0]], [0.25]), SPHERE_ONE, 0, 1.0)
    assert o["min_s2"][0] == 0.0 and o["band_kink"][0] == 1
    o = oracle.query(_scene([[0.75, 0, 0]], [0.25]), SPHERE_ONE, 0, 1.0)
    assert o["min_s2"][0] == pytest.approx(3 / 16, rel=1e-14) and o["band_kink"][0] == 0
    # relative to the terms: raw = 1e-6 against s^2 + n sqrt(sigma^2) = 1/4 + 1/4
    # is within 1e-5 (1/2); D = 1/2 + 2e-6 gives raw ~ 1e-6
    o = oracle.query(_scene([[0.5 + 2e-6, 0, 0]], [0.25]), SPHERE_ONE, 0, 1.0)
    assert 0 < o["min_s2"][0] < 2e-6 and o["band_kink"][0] == 1
    o = oracle.query(_scene([[0.5 + 4e-5, 0, 0]], [0.25]), SPHERE_ONE, 0, 1.0)
    assert o["min_s2"][0] > 1e-5 and o["band_kink"][0] == 0


# ------------------------------------------------------------------- gscale
def test_gscale_by_hand():
    """r = 1, n = 1, gamma = 5, s_min = 1, isotropic s = 1/4 at D = 2 on the
    +x and -x axes.  Each pair: s^2 = 4, sqrt(sigma^2) = 1, st^2 = 3 (in N_j,
    above s_min), dc = exp(-5 (3 - 1)) = e^-10.  d st^2/dc: the -2 d part has
    norm 4, the n sqrt(sigma^2) part 2 n Sigma d / sqrt(d^T Sigma d) has
    norm 2 (1/16)(2) / (1/2) = 1/2; so one pair's term size is
    gamma dc (4 + 1/2) = 22.5 e^-10.  The two pairs' gradients cancel
    exactly (mirror images), but their sizes add."""
    sc = _scene([[2, 0, 0], [-2, 0, 0]], [0.25])
    e10 = math.exp(-10.0)
    g, s = oracle.grad(sc, SPHERE_ONE, 0, 1.0, oracle.MODE_SUM, return_scale=True)
    assert np.abs(g).max() < 1e-20
    assert s[0] == pytest.approx(45 * e10, rel=1e-13)
    g, s = oracle.grad(sc, SPHERE_ONE, 0, 1.0, oracle.MODE_MEAN, return_scale=True)
    assert s[0] == pytest.approx(22.5 * e10, rel=1e-13)  # divided by |N_j| = 2
    g, s = oracle.grad(sc, SPHERE_ONE, 0, 1.0, oracle.MODE_MEAN, grad_out=[-2.0], return_scale=True)
    assert s[0] == pytest.approx(45 * e10, rel=1e-13)    # |upstream| scales it
    # min mode: the arg-min pair alone (both st^2 = 3: the first), no gamma dc
    g, s = oracle.grad(sc, SPHERE_ONE, 0, 1.0, oracle.MODE_MIN, return_scale=True)
    assert s[0] == pytest.approx(4.5, rel=1e-13)
    assert g[0] == pytest.approx([-3.5, 0, 0], rel=1e-13)  # -2 d + 1/2 along +x: d = (2, 0, 0)
    # softmin: equal weights 1/2 each
    g, s = oracle.grad(sc, SPHERE_ONE, 0, 1.0, oracle.MODE_SOFTMIN, return_scale=True)
    assert s[0] == pytest.approx(4.5, rel=1e-13)


def test_gscale_one_sided_pair():
    """A single pair of the case above: the summed-cost gradient is
    -gamma dc (-3.5, 0, 0) = 17.5 e^-10 along +x and its size 22.5 e^-10; a
    pair below s_min (flat Eq. 11) adds nothing to either."""
    e10 = math.exp(-10.0)
    sc = _scene([[2, 0, 0], [0, 0.5, 0]], [0.25, 0.0])  # the second: st^2 = 1/4 < s_min
    g, s = oracle.grad(sc, SPHERE_ONE, 0, 1.0, oracle.MODE_SUM, return_scale=True)
    assert g[0] == pytest.approx([17.5 * e10, 0, 0], rel=1e-13, abs=1e-30)
    assert s[0] == pytest.approx(22.5 * e10, rel=1e-13)
    g, s = oracle.grad(sc, SPHERE_ONE, 0, 1.0, oracle.MODE_MEAN, return_scale=True)
    assert s[0] == pytest.approx(11.25 * e10, rel=1e-13)  # |N_j| = 2


def test_gscale_zero_outside_the_clamp():
    """Where Eq. 8 clamps (raw <= 0) the term is zero and so is its size."""
    sc = _scene([[0.5, 0, 0]], [0.25])  # raw = 0 exactly (see the band_kink case)
    g, s = oracle.grad(sc, SPHERE_ONE, 0, 1.0, oracle.MODE_MIN, return_scale=True)
    assert s[0] == 0.0 and not g.any()


def test_cond_cost_skips_the_flat_part_of_eq11():
    """r = 1/2, n = 1, s_min = 1.  Cancellation matters to the cost only where
    Eq. 11 is not flat, st^2 >= s_min:
      G_p: s = 1/2 at (0, 1, 0): s^2 = 4, sqrt(sigma^2) = 2 (1/2)(1)/(1/4) = 4,
           st^2 = 0 (flat part), cond 8;
      G_q: s = 1/8 at (1, 0, 0): s^2 = 4, sqrt(sigma^2) = 2 (1/8)(1)/(1/4) = 1,
           st^2 = 3 (in N_j, above s_min), cond 5.
    cond = 8, cond_cost = 5; with s_min = 0 both count (cond_cost = 8); with
    only G_p, cond_cost = 0."""
    sc = _scene([[0, 1, 0], [1, 0, 0]], [0.5, 0.125])
    o = oracle.query(sc, SPHERE_HALF, 0, 1.0)
    assert o["count_nbr"][0] == 2
    assert o["cond"][0] == pytest.approx(8.0, rel=1e-14)
    assert o["cond_cost"][0] == pytest.approx(5.0, rel=1e-14)
    o = oracle.query(sc, SPHERE_HALF, 0, 1.0, oracle.Params(s_min=0.0))
    assert o["cond_cost"][0] == pytest.approx(8.0, rel=1e-14)
    o = oracle.query(_scene([[0, 1, 0]], [0.5]), SPHERE_HALF, 0, 1.0)
    assert o["cond"][0] == pytest.approx(8.0, rel=1e-14) and o["cond_cost"][0] == 0.0
    # just below s_min, within band (s^2 + n sqrt(sigma^2)) of it, still counts:
    # point Gaussians at st^2 = 1 - 0.5e-5 and 1 - 4e-5 against the unit sphere, n = 0
    o = oracle.query(_points_at_st2([1 - 0.5e-5]), SPHERE_ONE, 0, 0.0)
    assert o["cond_cost"][0] == pytest.approx(1 - 0.5e-5, rel=1e-6)
    o = oracle.query(_points_at_st2([1 - 4e-5]), SPHERE_ONE, 0, 0.0)
    assert o["cond_cost"][0] == 0.0
