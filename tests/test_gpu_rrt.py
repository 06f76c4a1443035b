"""cs_rrt_extend (batched RRT extension, tree on the device) against the RRT
oracle, extension by extension from the same tree.

Nearest nodes, new nodes and edge points are computed in FP32 by both sides
with the same correctly rounded operations, so they must agree bit for bit;
edge flags must agree exactly except for edges with a point whose pair sits
in the collision band (|st^2 - 1| <= 1e-5), which are counted; the grown tree
(nodes, parents, count) must then agree exactly.
"""
import numpy as np
import pytest

import cs_synth as S
from oracle import rrt as orrt

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cs(cuda_device):
    import paper_2609_35619_b300 as cs
    return cs


@pytest.fixture(scope="module")
def room(cs):
    sc = S.drone_scene(n=200_000)
    return sc, cs.Scene(sc["means"], sc["scales"], sc["quats"], sc["opacity"])


@pytest.mark.parametrize("ns,k_thr", [(1.0, 0), (0.0, 3)])
def test_extensions_match_oracle(cs, room, ns, k_thr):
    import oracle
    sc, scene = room
    d = orrt.RrtDesc(B=32, M=8, step=0.3, radius=0.05, nsigma=ns, capacity=512)
    # the root: the first of a few seeded points that the oracle finds free
    cand = np.random.default_rng(11).uniform([0.5, 0.5, 0.5], [5.5, 4.5, 2.5], (64, 3)).astype(np.float32)
    res = oracle.query(sc, np.c_[cand, np.full(64, d.radius, np.float32)], 0, ns, oracle.Params(k_thr=k_thr))
    root = cand[np.flatnonzero((res["collide"] == 0) & (res["band_in"] == 0))[0]]
    tree = cs.RrtTree(scene, root, capacity=d.capacity, step=d.step, radius=d.radius, nsigma=ns,
                      M=d.M, params=cs.QueryParams(k_thr=k_thr))
    nodes = np.zeros((d.capacity, 3), np.float32)
    nodes[0] = root
    parent = np.full(d.capacity, -1, np.int64)
    count = 1
    rng = np.random.default_rng(7 + k_thr)
    banded = inserted_free = collided = 0
    for it in range(6):
        samples = rng.uniform([0.1, 0.1, 0.1], [5.9, 4.9, 2.9], (d.B, 3)).astype(np.float32)
        out = tree.extend(samples)
        torch.cuda.synchronize()
        ref = orrt.extend(sc, nodes, parent, count, samples, d, oracle.Params(k_thr=k_thr))
        np.testing.assert_array_equal(out["nearest"].cpu().numpy(), ref["nearest"], err_msg=f"it {it}")
        free = out["edge_free"].cpu().numpy().astype(bool)
        band = ref["edge_band"]
        banded += int(band.sum())
        np.testing.assert_array_equal(free[~band], ref["edge_collide"][~band] == 0, err_msg=f"it {it}")
        if (free != (ref["edge_collide"] == 0)).any():
            break  # a band edge went the other way: the trees part here
        g_nodes = tree.nodes.cpu().numpy()
        g_parent = tree.parent.cpu().numpy()
        g_count = int(tree.count.cpu().item())
        assert g_count == ref["count"], it
        np.testing.assert_array_equal(g_nodes[:g_count], ref["nodes"][:g_count], err_msg=f"it {it}")
        np.testing.assert_array_equal(g_parent[:g_count], ref["parent"][:g_count], err_msg=f"it {it}")
        inserted_free += int(free.sum())
        collided += int((~free).sum())
        nodes, parent, count = ref["nodes"], ref["parent"], ref["count"]
    assert inserted_free > 0 and collided > 0, (inserted_free, collided)
    assert banded <= 2


def test_capacity_and_arguments(cs, room):
    _, scene = room
    tree = cs.RrtTree(scene, [3.0, 2.5, 1.5], capacity=5, step=0.2, radius=0.05, nsigma=0.0)
    rng = np.random.default_rng(3)
    for _ in range(4):
        tree.extend(rng.uniform([2.6, 2.1, 1.1], [3.4, 2.9, 1.9], (8, 3)).astype(np.float32))
    torch.cuda.synchronize()
    assert int(tree.count.item()) <= 5
    par = tree.parent.cpu().numpy()[: int(tree.count.item())]
    assert par[0] == -1 and (par[1:] >= 0).all() and (par[1:] < np.arange(1, len(par))).all()
    with pytest.raises(cs.CsError):
        bad = cs.RrtTree(scene, [3.0, 2.5, 1.5], capacity=5, step=-1.0)
        bad.extend(np.zeros((2, 3), np.float32))
    with pytest.raises(cs.CsError):
        tree.M = 1
        tree.extend(np.zeros((2, 3), np.float32))


def test_captured_extension_grows_the_same_tree(cs, room):
    """Replays of the captured extension (cs_rrt_graph_create), the samples
    rewritten before each launch, grow the same tree bit for bit as the same
    loop of cs_rrt_extend calls."""
    _, scene = room
    # the root: the first of a few seeded points that a query finds free
    cand = np.random.default_rng(11).uniform([0.5, 0.5, 0.5], [5.5, 4.5, 2.5], (64, 3)).astype(np.float32)
    res = scene.query(torch.as_tensor(np.c_[cand, np.full(64, 0.05, np.float32)], device="cuda"), 1.0)
    torch.cuda.synchronize()
    root = cand[np.flatnonzero(res["collide"].cpu().numpy() == 0)[0]]
    kw = dict(capacity=4096, step=0.3, radius=0.05, nsigma=1.0, M=8)
    a = cs.RrtTree(scene, root, **kw)
    b = cs.RrtTree(scene, root, **kw)
    g = b.graph(32)
    assert g.kernels > 0
    rng = np.random.default_rng(21)
    for _ in range(12):
        s = torch.as_tensor(rng.uniform([0.1, 0.1, 0.1], [5.9, 4.9, 2.9], (32, 3)).astype(np.float32), device="cuda")
        ra = a.extend(s)
        g.samples.copy_(s)
        g.launch()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(ra["nearest"].cpu().numpy(), g.nearest.cpu().numpy())
        np.testing.assert_array_equal(ra["edge_free"].cpu().numpy(), g.edge_free.cpu().numpy())
    n = int(a.count.item())
    assert n == int(b.count.item()) and n > 1
    np.testing.assert_array_equal(a.nodes[:n].cpu().numpy(), b.nodes[:n].cpu().numpy())
    np.testing.assert_array_equal(a.parent[:n].cpu().numpy(), b.parent[:n].cpu().numpy())
    g.close()
