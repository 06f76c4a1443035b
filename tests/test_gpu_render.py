"""cs_render (Section II-A, Eq. 3-4) against the FP64 rasterizer oracle,
pixel by pixel, through the C ABI.

Tolerance, per pixel and channel: every output moves by at most 2 T_k per
unit change of a Gaussian's alpha G (T_k its transmittance).  The FP32 value
of alpha_k G_k carries a relative error of at most c u (1 + q_k kappa_k),
where q_k is the quadratic form, kappa_k the condition number of Sigma'_k and
u = 2^-24.  Entries of Sigma' rounded by about 12 u of its largest eigenvalue
move q by up to 24 u q kappa; the conic and the three-term evaluation add
about 4 u q kappa more; halving for the exponent gives c = 16.  So
  |gpu - oracle| <= base = 2 c u cond + 8 u K + 1e-6
with cond = sum_k w_k (1 + q_k kappa_k) and K the number of blended Gaussians,
both from the oracle.  The depth output scales the same bound by the largest
distance.

A Gaussian whose alpha G lies within its error band of 1/255 may be drawn on
one side and not on the other; both results are valid.  Its effect, at most
2 (1/255) T_k, is added to the tolerance (the oracle's `slack`), and at most
1 % of the checked pixels may exceed the base bound.  Pixels whose stopping
test (transmittance near 1e-4) lies in its band, or whose order holds a depth
tie, are excluded and counted.
"""
import numpy as np
import pytest

import cs_synth as S
from oracle import raster

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
U32 = 2.0 ** -24
C = 16.0


@pytest.fixture(scope="module")
def cs(cuda_device):
    import paper_2609_35619_b300 as cs
    return cs


def _scene(cs, sc, colors, **kw):
    s = cs.Scene(sc["means"], sc["scales"], sc["quats"], sc.get("opacity"), **kw)
    s.set_appearance(sc.get("opacity"), colors)
    return s


def _compare(gpu, orc, label, pix=None, min_checked=0.9):
    """gpu: dict of numpy arrays (full images, or rows matching orc when pix is given)."""
    if pix is not None:
        v, x, y = pix[:, 0], pix[:, 1], pix[:, 2]
        g_rgb, g_dep, g_alp = gpu["rgb"][v, y, x], gpu["depth"][v, y, x], gpu["alpha"][v, y, x]
    else:
        g_rgb, g_dep, g_alp = gpu["rgb"], gpu["depth"], gpu["alpha"]
    ok = (orc["flags"] & 6) == 0
    base = 2 * C * U32 * orc["cond"] + 8 * U32 * orc["ncontrib"] + 1e-6
    tol = base + orc["slack"]
    dmax = max(float(np.abs(orc["depth"]).max()), 1.0)
    e_rgb = np.abs(g_rgb.astype(np.float64) - orc["rgb"]).max(-1)
    e_alp = np.abs(g_alp.astype(np.float64) - orc["alpha"])
    e_dep = np.abs(g_dep.astype(np.float64) - orc["depth"])
    over = np.zeros(ok.shape, bool)
    for name, e, t, b in (("rgb", e_rgb, tol, base), ("alpha", e_alp, tol, base),
                          ("depth", e_dep, tol * dmax, base * dmax)):
        bad = ok & (e > t)
        assert not bad.any(), (f"{label}: {bad.sum()}/{ok.sum()} {name} mismatches; worst "
                               f"{e[bad].max():.3e} vs tol {t[bad][np.argmax(e[bad])]:.3e}")
        over |= ok & (e > b)
    assert over.sum() <= 0.01 * ok.sum(), (label, int(over.sum()), int(ok.sum()))
    assert ok.mean() >= min_checked, (label, ok.mean())
    return {"pixels": int(ok.size), "excluded": int((~ok).sum()), "over_base": int(over.sum()),
            "max_err": float(e_rgb[ok].max())}


def _np(out):
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("dilation", [0.3, 0.0])
def test_small_scene_all_pixels(cs, dilation):
    """2,000 Gaussians in a 2 m cube, 6 views of 70 x 45 pixels (ragged
    tiles), background colour, every pixel against the oracle."""
    sc = S.tiny_scene(n=2000)
    col = S.scene_colors(sc)
    rng = np.random.default_rng(3)
    cams = np.stack([S.look_at(rng.uniform(-1.0, 3.0, 3) + [0, 0, 2.5], rng.uniform(0.5, 1.5, 3), f=60,
                               width=70, height=45) for _ in range(6)])
    scene = _scene(cs, sc, col)
    bg = (0.1, 0.2, 0.3)
    out = _np(scene.render(torch.as_tensor(cams, device="cuda"), 70, 45, dilation=dilation, background=bg))
    orc = raster.render(sc, col, cams, 70, 45, dilation=dilation, background=bg)
    rep = _compare(out, orc, f"small dil={dilation}")
    assert (orc["alpha"] > 0.5).mean() > 0.05 and (orc["alpha"] == 0).mean() > 0.01, rep


def test_disks_filter_and_near_plane(cs):
    """A 2DGS disk scene (singular Sigma: the dilation keeps Sigma' invertible)
    with the floater filter, seen from cameras inside the scene (Gaussians
    behind the camera and near the near plane)."""
    sc = S.tiny_scene(n=3000, seed=77)
    sc["scales"][:, 2] = 0.0
    sc["scales"][::50] *= 8.0          # some large ones, a few filtered as floaters
    col = S.scene_colors(sc, seed=5)
    rng = np.random.default_rng(4)
    cams = np.stack([S.look_at(rng.uniform(0.6, 1.4, 3), rng.uniform(0.0, 2.0, 3), f=40, width=48, height=40)
                     for _ in range(4)])
    scene = _scene(cs, sc, col)
    out = _np(scene.render(torch.as_tensor(cams, device="cuda"), 48, 40, near_plane=0.05))
    orc = raster.render(sc, col, cams, 48, 40, near_plane=0.05)
    _compare(out, orc, "disks inside the scene", min_checked=0.85)


def test_batch_equals_views_alone_and_repeats(cs):
    """Each view's image does not depend on the other views of the call, bit
    for bit, and a repeated call gives the same bits."""
    sc = S.tiny_scene(n=2000)
    col = S.scene_colors(sc)
    rng = np.random.default_rng(9)
    cams = np.stack([S.look_at(rng.uniform(-1.0, 3.0, 3) + [0, 0, 2.5], rng.uniform(0.5, 1.5, 3), f=50,
                               width=40, height=33) for _ in range(5)])
    scene = _scene(cs, sc, col)
    tc = torch.as_tensor(cams, device="cuda")
    a = _np(scene.render(tc, 40, 33))
    b = _np(scene.render(tc, 40, 33))
    for k in a:
        np.testing.assert_array_equal(a[k].view(np.uint32), b[k].view(np.uint32))
    for v in range(5):
        one = _np(scene.render(tc[v:v + 1], 40, 33))
        for k in a:
            np.testing.assert_array_equal(one[k][0].view(np.uint32), a[k][v].view(np.uint32))


def test_drone_room_terminal_views_sampled(cs):
    """The 500k-Gaussian drone room from 256 terminal states of MPPI rollouts,
    128 x 128 pixels, near plane 0.2 m, one call (the benchmark's launch);
    sampled pixels of a few views against the oracle."""
    sc = S.drone_scene()
    col = S.scene_colors(sc)
    cams = S.drone_terminal_cameras(rollouts=256)
    scene = _scene(cs, sc, col)
    out = _np(scene.render(torch.as_tensor(cams, device="cuda"), 128, 128, near_plane=0.2))
    rng = np.random.default_rng(12)
    views = rng.choice(256, 8, replace=False)
    pix = np.stack([np.repeat(views, 150), rng.integers(0, 128, 1200), rng.integers(0, 128, 1200)], 1)
    orc = raster.render(sc, col, cams, 128, 128, pixels=pix, near_plane=0.2)
    rep = _compare(out, orc, "drone room sample", pix=pix, min_checked=0.95)
    assert (orc["alpha"] > 0.5).mean() > 0.3, rep


def test_arguments_and_empty_cases(cs):
    sc = S.tiny_scene(n=500)
    scene = cs.Scene(sc["means"], sc["scales"], sc["quats"], sc["opacity"])
    cams = torch.as_tensor(S.look_at([1, 1, 4], [1, 1, 1], up=(0, 1, 0), f=30, width=20, height=20)[None],
                           device="cuda")
    with pytest.raises(cs.CsError):  # no appearance yet
        scene.render(cams, 20, 20)
    scene.set_appearance(sc["opacity"], S.scene_colors(sc))
    with pytest.raises(cs.CsError):
        scene.render(cams, 0, 20)
    with pytest.raises(cs.CsError):
        scene.render(cams, 20, 20, dilation=-1.0)
    out = scene.render(cams[:0], 20, 20)
    assert out["rgb"].shape == (0, 20, 20, 3)
    # a camera looking away from everything: background only
    away = torch.as_tensor(S.look_at([1, 1, 4], [1, 1, 9], up=(0, 1, 0), f=30, width=20, height=20)[None],
                           device="cuda")
    o = _np(scene.render(away, 20, 20, background=(0.25, 0.5, 0.75)))
    np.testing.assert_array_equal(o["alpha"], 0.0)
    np.testing.assert_array_equal(o["rgb"][0], np.broadcast_to(np.float32([0.25, 0.5, 0.75]), (20, 20, 3)))
    # an empty scene
    empty = cs.Scene(np.zeros((0, 3)), np.zeros((0, 3)), np.zeros((0, 4)))
    empty.set_appearance()
    o = _np(empty.render(cams, 20, 20, background=(0.5, 0.5, 0.5)))
    np.testing.assert_array_equal(o["rgb"], 0.5)
