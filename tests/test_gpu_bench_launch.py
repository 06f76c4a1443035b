"""The benchmark's timed launches, checked against the FP64 oracle at full
size: the 1M-Gaussian tabletop with the 262,144 arm spheres (groups of 64, one
per configuration) and the 2,097,152 RRT edge spheres (groups of 1,024, one per
edge), each as one conservatism-sweep call over n_sigma = 0, 0.5, 1, 2 on tile
shape 30 (the shape the autotuner picks for the benchmark: row quads, the sweep
copies sharing their geometry and evaluated as whole quads, k_thr = 0 flags as
one bit per row, four CTAs per SM, persistent); the other quad shapes (27, 28,
29) give the same bits at full size.

Per n_sigma block: a seeded sample of at least 192 rows (half uniform, half
among rows that touch the scene) element by element, and whole groups (two
arm configurations, one edge) through their group outputs, with the bound
derived in compare_groups (rows in the cutoff band take the oracle's range
over the band's memberships).  Section II-D sums the cost over links and
horizon; Section II-E ORs the flags over an edge.
"""
import numpy as np
import pytest

import cs_synth as S
import oracle
from _parity import compare, compare_groups, cutoff_interval, to_np

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

NSIGMAS = (0.0, 0.5, 1.0, 2.0)
TILE = 30


@pytest.fixture(scope="module")
def tabletop(cuda_device):
    import paper_2609_35619_b300 as cs
    sc = S.tabletop_scene()
    return cs, sc, cs.Scene(sc["means"], sc["scales"], sc["quats"], sc["opacity"])


@pytest.mark.parametrize("batch", ["arm", "edge"])
def test_benchmark_sweep_launch_full_size(tabletop, batch):
    cs, sc, scene = tabletop
    q = S.arm_queries() if batch == "arm" else S.edge_queries()
    G = 64 if batch == "arm" else 1024
    n_groups = 2 if batch == "arm" else 1
    Q = q.shape[0]
    ng = Q // G
    out = to_np(scene.query(torch.as_tensor(q), 0.0, want_count=True,
                            params=cs.QueryParams(group_size=G, tile_config=TILE, sweep=NSIGMAS)))
    torch.cuda.synchronize()
    assert out["metric"].shape == (len(NSIGMAS) * Q,) and out["group_metric"].shape == (len(NSIGMAS) * ng,)
    P = oracle.Params()
    rng = np.random.default_rng(1000 + G)
    for b, ns in enumerate(NSIGMAS):
        rows = {k: out[k][b * Q:(b + 1) * Q] for k in ("metric", "collide", "count")}
        # element by element on a sample of rows
        touching = np.flatnonzero(rows["count"] > 0)
        assert touching.size > 0
        idx = np.unique(np.r_[rng.choice(Q, 96, replace=False),
                              rng.choice(touching, min(96, touching.size), replace=False)])
        assert idx.size >= 192 or touching.size < 96
        orc = oracle.query(sc, q[idx], 0, ns, P)
        rep = compare({k: v[idx] for k, v in rows.items()}, orc, 0, P, f"{batch} ns={ns} sample")
        assert rep["checked"] >= 100, rep
        # whole groups: every row, then the group outputs
        cand = np.unique(touching // G)
        for g in rng.choice(cand, min(n_groups, cand.size), replace=False):
            gr = np.arange(g * G, (g + 1) * G)
            og = oracle.query(sc, q[gr], 0, ns, P)
            grows = {k: v[gr] for k, v in rows.items()}
            grep = compare(grows, og, 0, P, f"{batch} ns={ns} group {g} rows")
            band = np.flatnonzero(og["band_cut"] > 0)
            interval = None
            if band.size:
                lo, hi = cutoff_interval(sc, q[gr], 0, ns, P, band, oracle.MODE_MEAN)
                interval = (band, lo, hi)
            n = compare_groups(out["group_metric"][b * ng + g: b * ng + g + 1],
                               out["group_collide"][b * ng + g: b * ng + g + 1], grows["metric"], og, grep, G,
                               oracle.MODE_MEAN, f"{batch} ns={ns} group {g}", interval=interval)
            assert n == 1


@pytest.mark.parametrize("batch", ["arm", "edge"])
def test_quad_shapes_agree_at_full_size(tabletop, batch):
    """Shapes 27, 28 (persistent), 29 and 30 (persistent) run the same
    per-lane accumulation order, so the benchmark's sweep launches give the
    same bits on each of them (shape 30 is the benchmark's)."""
    cs, sc, scene = tabletop
    q = torch.as_tensor(S.arm_queries() if batch == "arm" else S.edge_queries())
    G = 64 if batch == "arm" else 1024
    outs = {}
    for tile in (27, 28, 29, 30):
        outs[tile] = to_np(scene.query(q, 0.0, want_count=True,
                                       params=cs.QueryParams(group_size=G, tile_config=tile, sweep=NSIGMAS)))
        torch.cuda.synchronize()
    for tile in (27, 28, 29):
        for k in outs[TILE]:
            np.testing.assert_array_equal(outs[tile][k].view(np.uint8), outs[TILE][k].view(np.uint8),
                                          err_msg=f"{batch} tile {tile} {k}")
    scene.sync()
