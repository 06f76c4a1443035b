"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Small cases cover every output and mode on scenes the oracle finishes in
seconds (several tiles and a ragged tail); the full-size workloads run in the
launch configuration the benchmark times and are checked on a seeded sample
of rows that the oracle evaluates one by one.
"""
import numpy as np
import pytest

import cs_synth as S
import oracle
from _parity import compare, compare_groups, cutoff_interval, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cs(cuda_device):
    import paper_2609_35619_b300 as cs
    return cs


def _scene(cs, sc, **kw):
    return cs.Scene(sc["means"], sc["scales"], sc["quats"], sc.get("opacity"), **kw)


def _run(cs, scene, prims, ns, prim_type=0, mode=0, nsq=None, **kw):
    params = cs.QueryParams(mode=mode, **kw)
    out = scene.query(torch.as_tensor(prims), ns, prim_type=prim_type, params=params, want_count=True,
                      nsigma_per_query=None if nsq is None else torch.as_tensor(nsq, dtype=torch.float32))
    torch.cuda.synchronize()
    return to_np(out)


def _oracle_params(**kw):
    return oracle.Params(**kw)


# ------------------------------------------------------------- config 1
@pytest.mark.parametrize("nsigma", [0.0, 0.5, 1.0, 2.0])
@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_tiny_scene_all_modes(cs, nsigma, mode):
    sc = S.tiny_scene()
    q = S.tiny_queries()
    scene = _scene(cs, sc)
    out = _run(cs, scene, q, nsigma, mode=mode)
    orc = oracle.query(sc, q, 0, nsigma)
    rep = compare(out, orc, mode, oracle.Params(), f"tiny ns={nsigma} mode={mode}")
    assert rep["checked"] > 0.9 * rep["Q"]


@pytest.mark.parametrize("cfg", list(range(1, 31)))
@pytest.mark.parametrize("Q", [1, 37, 1000, 5000])
def test_tile_configs_and_ragged_batches(cs, cfg, Q):
    """Every tile shape, batch sizes spanning one to many tiles with a ragged tail."""
    sc = S.tiny_scene(n=3000)
    rng = np.random.default_rng(Q)
    q = np.c_[rng.uniform(0, 2, (Q, 3)), rng.uniform(0.05, 0.3, Q)].astype(np.float32)
    scene = _scene(cs, sc)
    out = _run(cs, scene, q, 1.0, tile_config=cfg)
    compare(out, oracle.query(sc, q, 0, 1.0), 0, oracle.Params(), f"cfg={cfg} Q={Q}")


def test_per_query_nsigma_and_k_thr(cs):
    sc = S.tiny_scene()
    q = S.tiny_queries(q=700)
    rng = np.random.default_rng(3)
    ns = rng.uniform(0, 2.5, q.shape[0]).astype(np.float32)
    scene = _scene(cs, sc)
    for k_thr in (0, 3):
        out = _run(cs, scene, q, 0.0, nsq=ns, k_thr=k_thr)
        orc = oracle.query(sc, q, 0, ns.astype(np.float64), oracle.Params(k_thr=k_thr))
        compare(out, orc, 0, oracle.Params(), f"per-row n_sigma k_thr={k_thr}")


@pytest.mark.parametrize("axes", [(0.03, 0.2), (0.008, 0.06)])
@pytest.mark.parametrize("mode", [0, 2, 3])
def test_ellipsoids(cs, mode, axes):
    """Ellipsoids, including thin ones (semi-axes down to 8 mm: entries of A
    near 1.6e4, so d^T A d of a chunk's padding point overflows and must not
    turn into a neighbour)."""
    sc = S.tiny_scene()
    rng = np.random.default_rng(4)
    centres = rng.uniform(0, 2, (600, 3))
    e = S.ellipsoid_queries(5, centres, semi_lo=axes[0], semi_hi=axes[1])
    kappa = (e[:, 7:10].max(1) / e[:, 7:10].min(1)).astype(np.float64) ** 2
    # the FP32 rounding of d^T A d (24 u kappa cond) widens the bands in which a
    # neighbour or collision decision may flip
    cond = oracle.query(sc, e, 1, 1.0)["cond"]
    band = max(1e-5, 24 * 2.0 ** -24 * kappa.max() * max(cond.max(), 4.0))
    orc = oracle.query(sc, e, 1, 1.0, oracle.Params(band=band))
    scene = _scene(cs, sc)
    # thin ellipsoids against 2 cm Gaussians cancel strongly in Eq. 8, and the
    # widened band puts more pairs near s_min under cond_cost: 66 of the 600
    # rows (11 %) take the widened bound with semi-axes from 8 mm
    cap = 0.05 if axes[0] >= 0.03 else 0.15
    for cfg in (1, 2, 3, 4, 18, 23, 27, 28, 29, 30):
        out = _run(cs, scene, e, 1.0, prim_type=1, mode=mode, tile_config=cfg)
        rep = compare(out, orc, mode, oracle.Params(), f"ellipsoid mode={mode}", kappa=kappa, max_cancel=cap)
        assert rep["checked"] > 0.5 * rep["Q"], rep


def test_nondefault_metric_parameters(cs):
    sc = S.tiny_scene()
    q = S.tiny_queries()
    kw = dict(gamma=2.0, d_max=3.0, s_min=1.5, eps=1e-4, tau=0.2)
    scene = _scene(cs, sc)
    for mode in (0, 1, 3):
        out = _run(cs, scene, q, 1.0, mode=mode, **kw)
        compare(out, oracle.query(sc, q, 0, 1.0, oracle.Params(**kw)), mode, oracle.Params(**kw),
                f"params mode={mode}")


@pytest.mark.parametrize("s_min", [-1.0, -2.5, -10.0])
def test_negative_s_min(cs, s_min):
    """s_min below 0: Eq. 11 is then below d_max even at st^2 = 0, the cutoff
    S_cut = s_min + ln(1/eps)/gamma drops below 1 (-2.5) or below 0 (-10:
    no neighbours at all).  The packed cost path, which does not clamp st^2 at
    0, must still give the clamped answers where st^2 would be negative."""
    sc = S.tiny_scene()
    q = S.tiny_queries()
    q[:, 3] *= 3.0  # large spheres: many pairs with st^2 clamped to 0
    kw = dict(s_min=s_min)
    scene = _scene(cs, sc)
    for mode in (0, 1, 3):
        out = _run(cs, scene, q, 2.0, mode=mode, **kw)
        orc = oracle.query(sc, q, 0, 2.0, oracle.Params(**kw))
        compare(out, orc, mode, oracle.Params(**kw), f"s_min={s_min} mode={mode}")
        if s_min == -10.0:
            assert (out["count"] == 0).all() and (out["collide"] == 0).all()
        elif mode == 0:
            assert (orc["count_nbr"] > 0).mean() > 0.3


def test_group_outputs(cs):
    """Section II-D group sums and Section II-E group flags against the
    oracle's rows, with the bound derived in compare_groups: the rows' own
    parity bounds plus the rounding of the FP32 group sum (warp sums for
    G >= 32, in-order sums below), rows in the cutoff band taking the
    oracle's range over the band's memberships."""
    sc = S.tiny_scene()
    q = S.tiny_queries(q=1000)
    scene = _scene(cs, sc)
    P = oracle.Params()
    orc = oracle.query(sc, q, 0, 1.0, P)
    band = np.flatnonzero(orc["band_cut"] > 0)
    lo, hi = cutoff_interval(sc, q, 0, 1.0, P, band, oracle.MODE_MEAN)
    for G in (32, 64, 7, 1000):
        params = cs.QueryParams(group_size=G)
        out = to_np(scene.query(torch.as_tensor(q), 1.0, params=params, want_count=True))
        assert out["group_metric"].shape == ((q.shape[0] + G - 1) // G,)
        rep = compare(out, orc, 0, P, f"groups G={G} rows")
        n = compare_groups(out["group_metric"], out["group_collide"], out["metric"], orc, rep, G, oracle.MODE_MEAN,
                           f"groups G={G}", interval=(band, lo, hi))
        assert n == out["group_metric"].shape[0]
        # the group flag is the OR of the rows' flags, exactly
        ng = out["group_collide"].shape[0]
        rows_or = np.array([out["collide"][k * G:(k + 1) * G].max() for k in range(ng)])
        np.testing.assert_array_equal(out["group_collide"], rows_or)


# --------------------------------------------------------------- edge cases
def test_empty_batch_and_empty_scene(cs):
    sc = S.tiny_scene()
    scene = _scene(cs, sc)
    res = scene.query(torch.zeros((0, 4)), 1.0)
    assert res["metric"].numel() == 0
    empty = cs.Scene(np.zeros((0, 3)), np.zeros((0, 3)), np.zeros((0, 4)))
    assert empty.info()["n_kept"] == 0
    out = to_np(empty.query(torch.as_tensor(S.tiny_queries()), 1.0, want_count=True))
    assert (out["metric"] == 0).all() and (out["collide"] == 0).all() and (out["count"] == 0).all()
    out = to_np(empty.query(torch.as_tensor(S.tiny_queries()), 1.0,
                            params=cs.QueryParams(mode=2)))
    assert np.isinf(out["metric"]).all()


def test_all_filtered_and_invalid_rows(cs):
    n = 500
    rng = np.random.default_rng(6)
    sc = {"means": rng.uniform(0, 1, (n, 3)).astype(np.float32),
          "scales": np.full((n, 3), 0.2, np.float32),
          "quats": np.tile(np.float32([1, 0, 0, 0]), (n, 1)),
          "opacity": np.full(n, 0.01, np.float32)}
    scene = _scene(cs, sc)
    assert scene.info()["n_kept"] == 0
    sc["means"][:10] = np.nan
    sc["opacity"][:] = 0.9
    scene = _scene(cs, sc)
    inf = scene.info()
    assert inf["n_invalid"] == 10 and inf["n_kept"] == n - 10
    q = np.c_[rng.uniform(0, 1, (64, 3)), np.full(64, 0.1)].astype(np.float32)
    out = _run(cs, scene, q, 1.0)
    good = {k: v[10:] for k, v in sc.items()}
    compare(out, oracle.query(good, q, 0, 1.0), 0, oracle.Params(), "invalid gaussian rows")


def test_invalid_query_rows_reported(cs):
    sc = S.tiny_scene()
    scene = _scene(cs, sc)
    q = S.tiny_queries(q=100).copy()
    q[5, 3] = -1.0
    q[7, 0] = np.nan
    out = _run(cs, scene, q, 1.0)
    assert np.isnan(out["metric"][5]) and np.isnan(out["metric"][7]) and out["collide"][5] == 0
    with pytest.raises(cs.CsError) as ei:
        scene.sync()
    assert ei.value.status == cs.abi.CS_ERR_INVALID_ARG
    scene.sync()  # cleared
    keep = np.setdiff1d(np.arange(100), [5, 7])
    sub = {k: v[keep] for k, v in out.items()}
    compare(sub, oracle.query(sc, q[keep], 0, 1.0), 0, oracle.Params(), "valid rows beside invalid")


@pytest.mark.parametrize("tile,sweep", [(29, (0.0, 0.5, 1.0, 2.0)), (30, (0.0, 0.5, 1.0, 2.0)),
                                        (28, (2.0, 1.0, 0.0, 0.5, 3.0, 0.1, 1.5, 0.7))])
def test_sweep_whole_quads_with_invalid_rows(cs, tile, sweep):
    """A conservatism sweep with a multiple of four n_sigma values on the quad
    shapes runs the whole-quad evaluation: every row quad is four copies of one
    prepared sphere, and the copies of an invalid sphere (NaN centre, negative
    radius) form dead quads that are never evaluated.  Their rows come out as
    NaN (metric) and 0 (flag, count), the error word reports them, and every
    other row of every n_sigma block keeps the bits of its own call; a ragged
    last tile (1,003 primitives)."""
    sc = S.tiny_scene(n=3000)
    scene = _scene(cs, sc)
    rng = np.random.default_rng(93)
    Q, G = 1003, 10
    q = np.c_[rng.uniform(0, 2, (Q, 3)), rng.uniform(0.05, 0.25, Q)].astype(np.float32)
    bad = np.array([0, 5, 64, 333, 1002])
    q[bad[::2], 0] = np.nan
    q[bad[1::2], 3] = -1.0
    ng = (Q + G - 1) // G
    one = scene.query(torch.as_tensor(q), 0.0, want_count=True,
                      params=cs.QueryParams(group_size=G, sweep=sweep, tile_config=tile))
    torch.cuda.synchronize()
    with pytest.raises(cs.CsError) as ei:
        scene.sync()
    assert ei.value.status == cs.abi.CS_ERR_INVALID_ARG
    scene.sync()  # cleared
    for b, ns in enumerate(sweep):
        blk = {k: one[k][b * Q:(b + 1) * Q].cpu().numpy() for k in ("metric", "collide", "count")}
        assert np.isnan(blk["metric"][bad]).all() and (blk["collide"][bad] == 0).all() and (blk["count"][bad] == 0).all()
        sep = scene.query(torch.as_tensor(q), ns, want_count=True, params=cs.QueryParams(group_size=G))
        torch.cuda.synchronize()
        with pytest.raises(cs.CsError):
            scene.sync()
        scene.sync()
        for k in ("metric", "collide", "count"):
            np.testing.assert_array_equal(blk[k].view(np.uint8), sep[k].cpu().numpy().view(np.uint8),
                                          err_msg=f"{tile} {ns} {k}")
        for k in ("group_metric", "group_collide"):
            np.testing.assert_array_equal(one[k][b * ng:(b + 1) * ng].cpu().numpy().view(np.uint8),
                                          sep[k].cpu().numpy().view(np.uint8), err_msg=f"{tile} {ns} {k}")
        assert (blk["count"] > 0).any()


def test_degenerate_gaussians_and_far_queries(cs):
    """2DGS-style disks (a zero scale), zero-size points, identity-less zero
    quaternions, queries far outside the scene box."""
    rng = np.random.default_rng(7)
    n = 1500
    sc = S.tiny_scene(n=n)
    sc["scales"][:300, 2] = 0.0
    sc["scales"][300:400] = 0.0
    sc["quats"][400:450] = 0.0
    q = S.tiny_queries(q=300).copy()
    q[:20, :3] += 50.0
    q[20:40, :3] -= 3.0
    scene = _scene(cs, sc)
    for ns in (0.0, 1.5):
        out = _run(cs, scene, q, ns)
        compare(out, oracle.query(sc, q, 0, ns), 0, oracle.Params(), f"degenerate ns={ns}")


@pytest.mark.parametrize("kw", [dict(cell_size=0.02), dict(cell_size=5.0), dict(tier_quantile=0.5),
                                dict(tier_quantile=1.0), dict(use_filter=False)])
def test_scene_build_options(cs, kw):
    """Tiny cells (many rows), one cell, a large tier holding half the scene,
    no large tier, the floater filter off: the results do not change."""
    sc = S.tiny_scene()
    q = S.tiny_queries()
    scene = _scene(cs, sc, **kw)
    out = _run(cs, scene, q, 2.0)
    p = oracle.Params(use_filter=kw.get("use_filter", True))
    compare(out, oracle.query(sc, q, 0, 2.0, p), 0, p, f"build {kw}")


def test_repack_matches_eq2(cs):
    """The exported 48-byte records equal the oracle's Eq. 2 covariances, in
    grid order, and the index permutation covers the kept rows exactly once."""
    sc = S.tiny_scene(n=4000)
    scene = _scene(cs, sc)
    pos, cov, idx = (t.cpu().numpy() for t in scene.export())
    sig, keep = oracle.covariances(sc)
    assert sorted(idx.tolist()) == np.flatnonzero(keep).tolist()
    np.testing.assert_array_equal(pos[:, :3], sc["means"][idx])
    np.testing.assert_allclose(pos[:, 3], sc["scales"][idx].max(1), rtol=0)
    S_ = sig[idx]
    # each FP32 entry sums three products bounded by max(scale)^2 after a few
    # roundings: error <= 2e-6 max(scale)^2
    smax2 = sc["scales"][idx].astype(np.float64).max(1) ** 2
    want = np.stack([S_[:, 0, 0], S_[:, 1, 1], S_[:, 2, 2], 2 * S_[:, 0, 1], 2 * S_[:, 0, 2],
                     2 * S_[:, 1, 2]], 1)
    err = np.abs(cov[:, :6] - want)
    assert (err <= 2e-6 * smax2[:, None]).all(), err.max()
    inf = scene.info()
    assert inf["n_grid"] + inf["n_large"] == inf["n_kept"]


def test_alone_equals_in_the_mix(cs):
    """A row's result does not depend on which other rows share its launch
    (bitwise): every neighbour is visited in the same global order."""
    sc = S.tiny_scene()
    q = S.tiny_queries(q=2000)
    scene = _scene(cs, sc)
    full = _run(cs, scene, q, 1.0)
    rng = np.random.default_rng(8)
    sub = rng.choice(2000, 77, replace=False)
    part = _run(cs, scene, q[sub], 1.0)
    np.testing.assert_array_equal(part["metric"], full["metric"][sub])
    np.testing.assert_array_equal(part["count"], full["count"][sub])


def test_host_io_path_equals_device_path(cs):
    sc = S.tiny_scene()
    q = S.tiny_queries(q=900)
    scene = _scene(cs, sc)
    dev = _run(cs, scene, q, 1.0, group_size=32)
    p = cs.QueryParams(group_size=32).to_c()
    p.host_io = 1
    Q = q.shape[0]
    m = np.empty(Q, np.float32)
    c = np.empty(Q, np.uint8)
    cnt = np.empty(Q, np.int32)
    gm = np.empty((Q + 31) // 32, np.float32)
    gc = np.empty_like(gm, dtype=np.uint8)
    p.out_count = cnt.ctypes.data
    p.out_group_metric = gm.ctypes.data
    p.out_group_collide = gc.ctypes.data
    cs.check(cs.abi.cs_query(scene.handle, 0, q, Q, 1.0, m, c, p))
    np.testing.assert_array_equal(m, dev["metric"])
    np.testing.assert_array_equal(c, dev["collide"])
    np.testing.assert_array_equal(cnt, dev["count"])
    np.testing.assert_array_equal(gm, dev["group_metric"])


def test_pair_stats(cs):
    sc = S.tiny_scene()
    q = S.tiny_queries()
    scene = _scene(cs, sc)
    stats = torch.zeros(2, dtype=torch.int64, device="cuda")
    out = to_np(scene.query(torch.as_tensor(q), 1.0, want_count=True, pair_stats=stats))
    st = stats.cpu().numpy()
    assert st[1] == out["count"].sum()
    assert st[0] >= st[1] and st[0] <= q.shape[0] * sc["means"].shape[0]


def test_wait_timeout_selftest_leaves_context_usable(cs):
    assert cs.abi.cs_selftest_wait_timeout(2000, None) == cs.abi.CS_ERR_TIMEOUT
    sc = S.tiny_scene()
    q = S.tiny_queries()
    out = _run(cs, _scene(cs, sc), q, 1.0)
    compare(out, oracle.query(sc, q, 0, 1.0), 0, oracle.Params(), "after timeout self-test")


# ------------------------------------------------- full-size workloads
def _sample(Q, k, seed):
    return np.sort(np.random.default_rng(seed).choice(Q, size=min(k, Q), replace=False))


def test_drone_mppi_full_size(cs):
    """500k-Gaussian room, 1,024 rollouts x 32 steps, per-rollout outputs."""
    sc = S.drone_scene()
    q = S.drone_queries()
    scene = _scene(cs, sc)
    out = _run(cs, scene, q, 1.0, group_size=32)
    idx = _sample(q.shape[0], 192, 11)
    orc = oracle.query(sc, q[idx], 0, 1.0)
    rep = compare({k: v[idx] for k, v in out.items() if v.shape[0] == q.shape[0]}, orc, 0,
                  oracle.Params(), "drone sample")
    assert rep["checked"] > 100
    # group outputs are the sums of the per-row outputs
    np.testing.assert_allclose(out["group_metric"], out["metric"].reshape(-1, 32).astype(np.float64).sum(1),
                               rtol=1e-5)
    assert (out["group_collide"] == out["collide"].reshape(-1, 32).max(1)).all()


@pytest.mark.parametrize("nsigma", [0.0, 0.5, 1.0, 2.0])
def test_tabletop_full_size(cs, nsigma):
    """1M-Gaussian tabletop, 262,144 arm spheres + 2,097,152 RRT edge spheres
    in one launch (the benchmark's launch), sampled rows checked."""
    sc = _TABLE["scene"]
    q = _TABLE["queries"]
    scene = _TABLE.get("gpu") or _scene(cs, sc)
    _TABLE["gpu"] = scene
    out = _run(cs, scene, q, nsigma)
    idx = _sample(q.shape[0], 128, 12 + int(nsigma * 10))
    # bias the sample towards rows that touch the scene
    touching = np.flatnonzero(out["count"] > 0)
    idx2 = np.random.default_rng(13).choice(touching, size=min(64, touching.size), replace=False)
    idx = np.unique(np.r_[idx, idx2])
    orc = oracle.query(sc, q[idx], 0, nsigma)
    rep = compare({k: v[idx] for k, v in out.items()}, orc, 0, oracle.Params(), f"tabletop ns={nsigma}")
    assert rep["checked"] > 100


_TABLE = {}


@pytest.fixture(scope="module", autouse=True)
def _tabletop_data():
    _TABLE["scene"] = S.tabletop_scene()
    _TABLE["queries"] = np.concatenate([S.arm_queries(), S.edge_queries()])
    yield
    _TABLE.clear()


# ------------------------------------------------------ flags-only mode
@pytest.mark.parametrize("k_thr", [0, 3])
@pytest.mark.parametrize("prim_type", [0, 1])
def test_flags_mode_matches_full_evaluation_and_oracle(cs, k_thr, prim_type):
    """Flags mode (early exit): finished rows carry the same flag as the full
    evaluation (same FP32 decision), unfinished rows (2) only occur in
    colliding groups, group flags equal the full evaluation's and the
    oracle's (outside the collision band)."""
    sc = S.tiny_scene(n=3000)
    rng = np.random.default_rng(40 + k_thr)
    Q, G = 4000, 4
    c = rng.uniform(0, 2, (Q, 3))
    prims = (np.c_[c, rng.uniform(0.02, 0.06, Q)] if prim_type == 0
             else S.ellipsoid_queries(41, c, semi_lo=0.02, semi_hi=0.06)).astype(np.float32)
    scene = _scene(cs, sc)
    full = scene.query(torch.as_tensor(prims), 1.0, prim_type=prim_type,
                       params=cs.QueryParams(k_thr=k_thr, group_size=G))
    fl = scene.query(torch.as_tensor(prims), 1.0, prim_type=prim_type,
                     params=cs.QueryParams(k_thr=k_thr, group_size=G, mode=cs.CS_METRIC_FLAGS))
    torch.cuda.synchronize()
    f_row, g_row = fl["collide"].cpu().numpy(), full["collide"].cpu().numpy()
    done = f_row != 2
    np.testing.assert_array_equal(f_row[done], g_row[done])
    gf, gg = fl["group_collide"].cpu().numpy(), full["group_collide"].cpu().numpy()
    np.testing.assert_array_equal(gf, gg)
    assert (gg[np.flatnonzero(~done) // G] == 1).all(), "unfinished rows only in colliding groups"
    assert (~done).sum() > 0 and gg.sum() > 0 and (gg == 0).sum() > 0
    orc = oracle.query(sc, prims, prim_type, 1.0, oracle.Params(k_thr=k_thr))
    og = oracle.group_reduce(orc["mean_cost"], orc["collide"], G)[1]
    band = oracle.group_reduce(orc["mean_cost"], orc["band_in"] > 0, G)[1].astype(bool)
    np.testing.assert_array_equal(gf[~band], og[~band])


def test_flags_mode_without_groups_equals_full_flags(cs):
    sc = S.drone_scene(n=200_000)
    q = S.drone_queries(rollouts=512, horizon=32)
    scene = _scene(cs, sc)
    full = scene.query(torch.as_tensor(q), 1.0)
    fl = scene.query(torch.as_tensor(q), 1.0, params=cs.QueryParams(mode=cs.CS_METRIC_FLAGS))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(fl["collide"].cpu().numpy(), full["collide"].cpu().numpy())


def test_nsigma_sweep_in_one_launch_equals_separate_launches(cs):
    """The arm batch at four n_sigma values in one launch (rows repeated,
    n_sigma per row, as the benchmark runs the sweep) gives every row the same
    bits as four separate launches, in every metric mode."""
    sc = _TABLE["scene"]
    q = S.arm_queries(configs=1024)
    scene = _TABLE.get("gpu") or _scene(cs, sc)
    _TABLE["gpu"] = scene
    ns = np.array([0.0, 0.5, 1.0, 2.0], np.float32)
    Q = q.shape[0]
    rows = torch.as_tensor(np.tile(q, (4, 1)), device="cuda")
    nsq = torch.as_tensor(np.repeat(ns, Q), device="cuda")
    for mode in (0, 2, 3):
        p = cs.QueryParams(mode=mode, group_size=64)
        one = scene.query(rows, 0.0, params=p, nsigma_per_query=nsq, want_count=True)
        for i, v in enumerate(ns):
            sep = scene.query(torch.as_tensor(q, device="cuda"), float(v), params=p, want_count=True)
            torch.cuda.synchronize()
            for k in ("metric", "collide", "count"):
                a = one[k][i * Q:(i + 1) * Q].cpu().numpy()
                b = sep[k].cpu().numpy()
                np.testing.assert_array_equal(a.view(np.uint8), b.view(np.uint8), err_msg=f"{mode} {v} {k}")
            np.testing.assert_array_equal(one["group_metric"][i * (Q // 64):(i + 1) * (Q // 64)].cpu().numpy(),
                                          sep["group_metric"].cpu().numpy())


@pytest.mark.parametrize("prim_type,tile,sweep,k_thr", [
    (0, 0, (0.0, 0.5, 1.0, 2.0, 1.25), 0), (1, 0, (0.0, 0.5, 1.0, 2.0, 1.25), 0),
    # the shapes whose sweep launches share geometry over row pairs (18, 22)
    # or row quads (15, 23-27), with copies aligned to the quads (four
    # values) or not (three, five)
    (0, 15, (0.0, 0.5, 1.0, 2.0), 0), (0, 18, (0.0, 0.5, 1.0, 2.0), 0), (0, 24, (0.0, 0.5, 1.0, 2.0), 0),
    (0, 24, (0.0, 0.5, 1.0, 2.0, 1.25), 0), (0, 24, (2.0, 0.0, 1.0), 0), (0, 23, (0.0, 0.5, 1.0, 2.0), 0),
    (0, 22, (0.0, 0.5, 1.0, 2.0), 0), (0, 15, (1.0, 0.5, 0.0), 0),
    # quads evaluated as one group of four, with one reach test per quad (25-30)
    (0, 26, (0.0, 0.5, 1.0, 2.0), 0), (0, 26, (0.0, 0.5, 1.0, 2.0, 1.25), 0), (0, 26, (2.0, 0.0, 1.0), 0),
    (0, 27, (0.0, 0.5, 1.0, 2.0), 0), (0, 27, (1.0, 0.5, 0.0), 0), (0, 26, (0.0, 0.5, 1.0, 2.0), 2),
    (0, 29, (0.0, 0.5, 1.0, 2.0), 0), (0, 29, (2.0, 0.0, 1.0), 0), (0, 29, (0.0, 0.5, 1.0, 2.0, 1.25), 2),
    (0, 30, (0.0, 0.5, 1.0, 2.0), 0),
    # eight values: two whole quads per primitive (the quad-only evaluation)
    (0, 29, (0.0, 0.25, 0.5, 0.75, 1.0, 1.5, 2.0, 3.0), 0), (0, 28, (2.0, 1.0, 0.0, 0.5, 3.0, 0.1, 1.5, 0.7), 1),
    (0, 25, (0.0, 0.5, 1.0, 2.0), 0), (0, 25, (0.0, 0.5, 1.0, 2.0, 1.25), 0), (0, 25, (2.0, 0.0, 1.0), 0),
    # k_thr > 0: in-collision counts instead of the smallest st^2
    (0, 25, (0.0, 0.5, 1.0, 2.0), 2), (0, 24, (0.0, 0.5, 1.0, 2.0), 1), (0, 0, (0.0, 1.0, 2.0), 3)])
def test_sweep_parameter_equals_separate_calls(cs, prim_type, tile, sweep, k_thr):
    """cs_params.sweep_count: one call over Q rows at S n_sigma values gives
    block s exactly the bits of its own call (metric, flag, count, groups
    within each block, with a ragged last group), in every metric mode."""
    sc = S.tiny_scene(n=3000)
    scene = _scene(cs, sc)
    rng = np.random.default_rng(90 + prim_type)
    Q, G = 1003, 10
    c = rng.uniform(0, 2, (Q, 3))
    q = (np.c_[c, rng.uniform(0.05, 0.25, Q)] if prim_type == 0
         else S.ellipsoid_queries(91, c, semi_lo=0.04, semi_hi=0.2)).astype(np.float32)
    q[::97] = q[1::97]  # some primitives repeated within the batch
    ng = (Q + G - 1) // G
    for mode in (0, 1, 2, 3):
        one = scene.query(torch.as_tensor(q), 0.0, prim_type=prim_type, want_count=True,
                          params=cs.QueryParams(mode=mode, group_size=G, sweep=sweep, tile_config=tile,
                                                k_thr=k_thr))
        torch.cuda.synchronize()
        assert one["metric"].shape[0] == len(sweep) * Q and one["group_metric"].shape[0] == len(sweep) * ng
        for s, ns in enumerate(sweep):
            sep = scene.query(torch.as_tensor(q), ns, prim_type=prim_type, want_count=True,
                              params=cs.QueryParams(mode=mode, group_size=G, k_thr=k_thr))
            torch.cuda.synchronize()
            for k in ("metric", "collide", "count"):
                np.testing.assert_array_equal(one[k][s * Q:(s + 1) * Q].cpu().numpy().view(np.uint8),
                                              sep[k].cpu().numpy().view(np.uint8), err_msg=f"{mode} {ns} {k}")
            for k in ("group_metric", "group_collide"):
                np.testing.assert_array_equal(one[k][s * ng:(s + 1) * ng].cpu().numpy().view(np.uint8),
                                              sep[k].cpu().numpy().view(np.uint8), err_msg=f"{mode} {ns} {k}")
    with pytest.raises(cs.CsError):  # no adjoint for a sweep
        scene.query_grad(torch.as_tensor(q), 0.0, prim_type=prim_type, params=cs.QueryParams(sweep=sweep))
    with pytest.raises(cs.CsError):  # no flags mode for a sweep
        scene.query(torch.as_tensor(q), 0.0, prim_type=prim_type,
                    params=cs.QueryParams(mode=cs.CS_METRIC_FLAGS, sweep=sweep))


@pytest.mark.parametrize("base,persistent", [(27, 28), (29, 30)])
def test_persistent_shape_equals_its_one_tile_per_cta_shape(cs, base, persistent):
    """Shapes 28 and 30 run shapes 27 and 29 as persistent kernels (SMs x 3
    or 4 CTAs taking tiles from a counter).  On a batch of far more tiles than the grid holds,
    with a ragged last tile, every output has the bits of its base shape: each row's
    reductions do not depend on which CTA or in which order its tile ran.
    Also as a conservatism sweep with groups, and twice in a row on one stream
    (the tile counter starts every launch at zero)."""
    sc = _TABLE["scene"]
    scene = _TABLE.get("gpu") or _scene(cs, sc)
    _TABLE["gpu"] = scene
    q = torch.as_tensor(S.edge_queries(edges=600)[:-13].copy())  # 153,587 rows: ~2,400 tiles of 64
    for params in ({}, {"group_size": 64, "sweep": (0.0, 0.5, 1.0, 2.0)}):
        ref = to_np(scene.query(q, 1.0, want_count=True, params=cs.QueryParams(tile_config=base, **params)))
        for rep in range(2):
            got = to_np(scene.query(q, 1.0, want_count=True, params=cs.QueryParams(tile_config=persistent, **params)))
            torch.cuda.synchronize()
            for k in ref:
                np.testing.assert_array_equal(got[k].view(np.uint8), ref[k].view(np.uint8), err_msg=f"{k} {params}")
        assert (ref["count"] > 0).any()
    scene.sync()
