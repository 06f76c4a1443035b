"""Pins of the rasterizer oracle (oracle/raster.py, Eq. 3-4) against values
fixed outside it: closed forms for Gaussians on the optical axis, the order
and stopping rules of Eq. 4 worked by hand, moments of the image of one
Gaussian against a Monte Carlo projection of samples through the pinhole
model, and the invariance of an image under a rigid motion of scene and
camera together."""
import math

import numpy as np

import cs_synth as S
from oracle import raster

THR = 1.0 / 255.0


def _scene(means, scales, quats=None, opacity=None):
    n = len(means)
    return {"means": np.asarray(means, np.float32).reshape(n, 3),
            "scales": np.asarray(scales, np.float32).reshape(n, 3),
            "quats": np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)) if quats is None
            else np.asarray(quats, np.float32).reshape(n, 4),
            "opacity": np.ones(n, np.float32) if opacity is None else np.asarray(opacity, np.float32)}


def _axis_cam(f=50.0, w=40, h=30, cx=None, cy=None):
    """Identity camera at the origin looking along +z (x right, y down)."""
    cx = w / 2.0 if cx is None else cx
    cy = h / 2.0 if cy is None else cy
    return np.array([1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0, f, f, cx, cy], np.float32)[None]


def test_single_gaussian_on_axis_closed_form():
    # isotropic std s at depth z on the axis: Sigma' = ((f s / z)^2 + dil) I,
    # a(x) = alpha exp(-|x - c|^2 / (2 s'^2)), zero where below 1/255
    s, z, f, dil, alpha = 0.05, 2.0, 50.0, 0.3, 0.8
    w, h = 40, 30
    sc = _scene([[0, 0, z]], [[s, s, s]], opacity=[alpha])
    col = np.array([[0.2, 0.5, 0.9]])
    out = raster.render(sc, col, _axis_cam(f, w, h), w, h, dilation=dil, use_filter=False)
    s32, z32 = float(np.float32(s)), float(np.float32(z))
    sp2 = (f * s32 / z32) ** 2 + dil
    yy, xx = np.mgrid[0:h, 0:w]
    r2 = (xx + 0.5 - w / 2) ** 2 + (yy + 0.5 - h / 2) ** 2
    a = float(np.float32(alpha)) * np.exp(-r2 / (2 * sp2))
    a = np.where(a >= THR, np.minimum(a, 0.99), 0.0)
    np.testing.assert_allclose(out["alpha"][0], a, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(out["rgb"][0], a[..., None] * col[0], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(out["depth"][0], a * z32, rtol=1e-12, atol=1e-15)
    assert (a == 0).any() and (a > 0).sum() > 20


def test_depth_output_is_the_distance_of_the_mean():
    # an off-axis Gaussian: the blended depth is |x_c| a, not z a
    m = np.array([0.3, -0.2, 1.5], np.float32)
    sc = _scene([m], [[0.04] * 3], opacity=[0.9])
    out = raster.render(sc, np.ones((1, 3)), _axis_cam(), 40, 30, use_filter=False)
    a = out["alpha"][0]
    k = np.unravel_index(np.argmax(a), a.shape)
    np.testing.assert_allclose(out["depth"][0][k], np.linalg.norm(m.astype(np.float64)) * a[k], rtol=1e-12)


def test_two_gaussians_blend_front_to_back():
    # both on the axis, centre pixel (G = 1 up to the half-pixel offset,
    # identical for both): c = c1 a1 + c2 a2 (1 - a1), nearer first
    sc = _scene([[0, 0, 1.0], [0, 0, 2.0]], [[0.05] * 3, [0.1] * 3], opacity=[0.6, 0.7])
    col = np.array([[1.0, 0, 0], [0, 1.0, 0]])
    cam = _axis_cam(w=41, h=41, cx=20.5, cy=20.5)
    out = raster.render(sc, col, cam, 41, 41, use_filter=False)
    rev = raster.render({k: v[::-1].copy() for k, v in sc.items()}, col[::-1].copy(), cam, 41, 41, use_filter=False)
    np.testing.assert_array_equal(out["rgb"], rev["rgb"])  # input order does not matter
    a1, a2 = float(np.float32(0.6)), float(np.float32(0.7))
    np.testing.assert_allclose(out["rgb"][0, 20, 20], [a1, a2 * (1 - a1), 0], rtol=1e-12)
    np.testing.assert_allclose(out["alpha"][0, 20, 20], 1 - (1 - a1) * (1 - a2), rtol=1e-12)
    # the red one moved behind: roles swap
    sc2 = _scene([[0, 0, 3.0], [0, 0, 2.0]], [[0.15] * 3, [0.1] * 3], opacity=[0.6, 0.7])
    out2 = raster.render(sc2, col, cam, 41, 41, use_filter=False)
    np.testing.assert_allclose(out2["rgb"][0, 20, 20], [a1 * (1 - a2), a2, 0], rtol=1e-12)


def test_clamp_and_early_stop():
    # centre pixel: a1 = min(1, 0.99) -> T = 0.01; a2 = 0.98 -> T = 2e-4;
    # a3 = 0.99 would bring T to 2e-6 < 1e-4: blending stops before it
    sc = _scene([[0, 0, 1.0], [0, 0, 1.5], [0, 0, 2.0]], [[0.05] * 3] * 3, opacity=[1.0, 0.98, 1.0])
    col = np.array([[1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0]])
    out = raster.render(sc, col, _axis_cam(w=41, h=41, cx=20.5, cy=20.5), 41, 41, use_filter=False,
                        background=(0.5, 0.5, 0.5))
    a2 = float(np.float32(0.98))
    T = 0.01 * (1 - a2)
    np.testing.assert_allclose(out["rgb"][0, 20, 20], [0.99 + 0.5 * T, a2 * 0.01 + 0.5 * T, 0.5 * T], rtol=1e-12)
    np.testing.assert_allclose(out["alpha"][0, 20, 20], 1 - T, rtol=1e-9)
    assert out["ncontrib"][0, 20, 20] == 2


def test_threshold_background_and_near_plane():
    bg = (0.1, 0.2, 0.3)
    # a faint Gaussian (alpha below 1/255) draws nothing anywhere
    faint = _scene([[0, 0, 1.0]], [[0.2] * 3], opacity=[0.0039])
    out = raster.render(faint, np.ones((1, 3)), _axis_cam(), 40, 30, background=bg, use_filter=False)
    np.testing.assert_array_equal(out["alpha"], 0.0)
    np.testing.assert_allclose(out["rgb"][0], np.broadcast_to(bg, (30, 40, 3)), rtol=0, atol=0)
    # behind the near plane or behind the camera: nothing
    for z in (0.005, -1.0):
        sc = _scene([[0, 0, z]], [[0.01] * 3], opacity=[0.9])
        out = raster.render(sc, np.ones((1, 3)), _axis_cam(), 40, 30, near_plane=0.01, use_filter=False)
        np.testing.assert_array_equal(out["alpha"], 0.0)


def _truncated_cov_factor(Q):
    # covariance of a 2D Gaussian restricted to its ellipse q <= Q, relative
    # to the full covariance (radial integral of the truncated density)
    e = math.exp(-Q / 2)
    return (1 - e * (1 + Q / 2)) / (1 - e)


def test_projection_moments_match_monte_carlo():
    """The image of one anisotropic, rotated Gaussian seen off axis from a
    rotated camera: its first and second moments over the pixels match the
    mean and covariance of 3D samples pushed through the pinhole model
    (no Jacobian involved), within the linearisation and Monte Carlo error."""
    rng = np.random.default_rng(5)
    w, h, f = 280, 240, 400.0
    # the mean projects well off the image centre in both directions, where
    # every entry of the Jacobian matters
    cam = S.look_at([0.3, -2.5, 1.2], [-0.25, 0.25, 0.0], f=f, width=w, height=h)[None]
    q = S.random_quats(rng, 1).astype(np.float32)
    mean = np.array([[0.15, 0.25, 0.35]], np.float32)
    scale = np.array([[0.06, 0.03, 0.015]], np.float32)
    alpha = 0.98
    sc = _scene(mean, scale, q, [alpha])
    out = raster.render(sc, np.ones((1, 3)), cam, w, h, dilation=0.0, use_filter=False)
    a = out["alpha"][0]
    yy, xx = np.mgrid[0:h, 0:w]
    px, py = xx + 0.5, yy + 0.5
    W = a / a.sum()
    mu_img = np.array([(W * px).sum(), (W * py).sum()])
    d = np.stack([px - mu_img[0], py - mu_img[1]])
    cov_img = np.einsum("iyx,jyx,yx->ij", d, d, W)
    # Monte Carlo through the pinhole model
    import oracle
    Sig, _ = oracle.covariances(sc, oracle.Params(use_filter=False))
    X = rng.multivariate_normal(mean[0].astype(np.float64), Sig[0], size=1_000_000)
    R = cam[0, :9].astype(np.float64).reshape(3, 3)
    t = cam[0, 9:12].astype(np.float64)
    Xc = X @ R.T + t
    uv = np.stack([f * Xc[:, 0] / Xc[:, 2] + w / 2, f * Xc[:, 1] / Xc[:, 2] + h / 2], 1)
    cov_mc = np.cov(uv.T)
    # the image keeps alpha G >= 1/255 only: the ellipse q <= 2 ln(255 alpha)
    fac = _truncated_cov_factor(2 * math.log(255 * alpha))
    np.testing.assert_allclose(mu_img, uv.mean(0), atol=0.05)
    np.testing.assert_allclose(cov_img, fac * cov_mc, rtol=0.02, atol=0.02 * np.abs(cov_mc).max())
    assert cov_mc[0, 0] > 20 and abs(cov_mc[0, 1]) > 1  # large and tilted enough to mean something
    off = uv.mean(0) - [w / 2, h / 2]
    assert (np.abs(off) > 30).all(), off


def test_rigid_motion_of_scene_and_camera_leaves_the_image():
    sc = S.tiny_scene(n=150)
    col = S.scene_colors(sc)
    cam = S.look_at([1.0, -1.5, 2.5], [1.0, 1.0, 1.0], f=30, width=24, height=20)
    out = raster.render(sc, col, cam[None], 24, 20, use_filter=False)
    # rotate everything by Q about the origin and shift by b
    rng = np.random.default_rng(8)
    qr = S.random_quats(rng, 1)[0]
    from scipy.spatial.transform import Rotation
    Q = Rotation.from_quat([qr[1], qr[2], qr[3], qr[0]])
    b = np.array([0.3, -0.7, 0.2])
    moved = dict(sc)
    moved["means"] = (Q.apply(sc["means"].astype(np.float64)) + b).astype(np.float32)
    qs = sc["quats"].astype(np.float64)
    comp = Q * Rotation.from_quat(np.c_[qs[:, 1:], qs[:, :1]])
    qq = comp.as_quat()
    moved["quats"] = np.c_[qq[:, 3:], qq[:, :3]].astype(np.float32)
    R = cam[:9].astype(np.float64).reshape(3, 3)
    t = cam[9:12].astype(np.float64)
    R2 = R @ Q.as_matrix().T
    t2 = t - R2 @ b
    cam2 = np.concatenate([R2.ravel(), t2, cam[12:]]).astype(np.float32)
    out2 = raster.render(moved, col, cam2[None], 24, 20, use_filter=False)
    assert out["alpha"].max() > 0.5
    np.testing.assert_allclose(out2["rgb"], out["rgb"], atol=2e-4)
    np.testing.assert_allclose(out2["alpha"], out["alpha"], atol=2e-4)
