"""Pins of the oracle's exact-variance option against values fixed outside
the oracle: the closed form for an isotropic Gaussian, a Monte Carlo
estimate of the variance of the quadratic form of Eq. 5 under the Gaussian
(the quantity Eq. 7 linearises), the ordering with the linearised variance,
and the gradient against central differences."""
import math

import numpy as np

import oracle
import cs_synth as S

EXACT = oracle.Params(exact_variance=True)


def test_isotropic_closed_form():
    # Sigma = s^2 I, sphere radius r (A = I / r^2), distance D:
    # var = 4 s^2 D^2 / r^4 + 2 tr(Sigma^2 / r^4) = (4 s^2 D^2 + 6 s^4) / r^4
    s, r, D, n = 0.05, 0.2, 0.3, 1.5
    q = np.array([1, 0, 0, 0], np.float32)
    mean = np.array([D, 0, 0], np.float32)
    prim = np.array([0, 0, 0, r], np.float32)
    sd, rd, Dd = float(np.float32(s)), float(np.float32(r)), float(np.float32(D))
    t = oracle.pair(mean, np.full(3, s, np.float32), q, prim, 0, n, EXACT)
    var = (4 * sd * sd * Dd * Dd + 6 * sd ** 4) / rd ** 4
    np.testing.assert_allclose(t["var"], var, rtol=1e-12)
    np.testing.assert_allclose(t["st2"], max(0.0, Dd * Dd / (rd * rd) - n * math.sqrt(var)), rtol=1e-12)
    lin = oracle.pair(mean, np.full(3, s, np.float32), q, prim, 0, n)
    np.testing.assert_allclose(lin["var"], 4 * sd * sd * Dd * Dd / rd ** 4, rtol=1e-12)


def _monte_carlo_var(mean, Sig, c, A, n=2_000_000, seed=0):
    rng = np.random.default_rng(seed)
    L = np.linalg.cholesky(Sig)
    X = mean + rng.standard_normal((n, 3)) @ L.T
    d = X - c
    s2 = np.einsum("ni,ij,nj->n", d, A, d)
    return s2.var()


def test_variance_matches_monte_carlo_for_an_ellipsoid():
    # an anisotropic Gaussian close to a thin rotated ellipsoid, where the
    # trace term matters: the oracle's exact variance is the sample variance
    # of s^2(X), X ~ N(mu, Sigma), within Monte Carlo error; the linearised
    # variance of Eq. 7 is not
    rng = np.random.default_rng(3)
    quat_g = S.random_quats(rng, 1)[0].astype(np.float32)
    scale = np.array([0.06, 0.03, 0.01], np.float32)
    mean = np.array([0.12, -0.05, 0.04], np.float32)
    prim = np.r_[np.zeros(3), S.random_quats(rng, 1)[0], [0.08, 0.05, 0.03]].astype(np.float32)
    Sig, _ = oracle.covariances({"means": mean[None], "scales": scale[None], "quats": quat_g[None],
                                 "opacity": np.ones(1, np.float32)}, oracle.Params(use_filter=False))
    # A from scipy (independent of the oracle's quaternion code)
    from scipy.spatial.transform import Rotation
    R = Rotation.from_quat(np.r_[prim[4:7], prim[3]].astype(np.float64)).as_matrix()
    A = R @ np.diag(1.0 / prim[7:10].astype(np.float64) ** 2) @ R.T
    mc = _monte_carlo_var(mean.astype(np.float64), Sig[0], np.zeros(3), A)
    ex = oracle.pair(mean, scale, quat_g, prim, 1, 1.0, EXACT)["var"]
    lin = oracle.pair(mean, scale, quat_g, prim, 1, 1.0)["var"]
    assert abs(ex - mc) / mc < 0.02, (ex, mc)
    assert abs(lin - mc) / mc > 0.05, (lin, mc)


def test_exact_variance_is_more_conservative():
    sc = S.tiny_scene(n=400)
    q = S.tiny_queries(q=64)
    a = oracle.query(sc, q, 0, 1.0)
    b = oracle.query(sc, q, 0, 1.0, EXACT)
    # a larger variance can only lower st^2: more neighbours, smaller minimum
    assert (b["count_nbr"] >= a["count_nbr"]).all() and (b["count_in"] >= a["count_in"]).all()
    assert (b["min_s2"][a["count_nbr"] > 0] <= a["min_s2"][a["count_nbr"] > 0] + 1e-12).all()
    assert (b["min_s2"][a["count_nbr"] > 0] < a["min_s2"][a["count_nbr"] > 0]).any()
    # n_sigma = 0: the variance plays no part
    np.testing.assert_array_equal(oracle.query(sc, q, 0, 0.0, EXACT)["count_nbr"],
                                  oracle.query(sc, q, 0, 0.0)["count_nbr"])


def test_exact_variance_gradient_against_central_differences():
    # the oracle's analytic gradient with the exact variance against central
    # differences of its own metric (float32 offsets, the step measured after
    # rounding), on queries whose neighbour sets stay put within the stencil
    rng = np.random.default_rng(21)
    sc = S.tiny_scene(n=600)
    Q = 30
    for ptype in (0, 1):
        c = rng.uniform(0.3, 1.7, (Q, 3))
        prims = (np.c_[c, rng.uniform(0.1, 0.25, Q)] if ptype == 0
                 else S.ellipsoid_queries(8, c, semi_lo=0.08, semi_hi=0.2)).astype(np.float32)
        h = 2e-4
        ga = oracle.grad(sc, prims, ptype, 1.0, oracle.MODE_SUM, params=EXACT)
        gf = np.zeros_like(ga)
        ok = np.ones(Q, bool)
        base = oracle.query(sc, prims, ptype, 1.0, EXACT)
        for a in range(3):
            pp, pm = prims.astype(np.float64).copy(), prims.astype(np.float64).copy()
            pp[:, a] += h
            pm[:, a] -= h
            pp32, pm32 = pp.astype(np.float32), pm.astype(np.float32)
            step = pp32[:, a].astype(np.float64) - pm32[:, a].astype(np.float64)
            rp, rm = oracle.query(sc, pp32, ptype, 1.0, EXACT), oracle.query(sc, pm32, ptype, 1.0, EXACT)
            gf[:, a] = (rp["sum_cost"] - rm["sum_cost"]) / step
            for r in (rp, rm):
                ok &= (r["count_nbr"] == base["count_nbr"]) & (r["count_in"] == base["count_in"])
        assert ok.sum() >= Q // 3
        scale = np.abs(ga[ok]).max() + 1e-12
        err = np.linalg.norm(ga[ok] - gf[ok], axis=1)
        assert (err <= 2e-3 * np.linalg.norm(ga[ok], axis=1) + 1e-4 * scale).all(), (ptype, err.max())
