"""Serving loop (cs_server_*): continuous batching over resident scenes.

Each request's results must be the same alone and in the mix: the server
answers requests of uneven size, for two scenes, with per-request n_sigma and
group sizes, submitted from several threads so that they share batches, and
every result must equal, bit for bit, a cs_query call on that request alone
(the fused kernel reduces each primitive in a fixed order whatever rows
share the launch).  A sample is also checked against the FP64 oracle.
"""
import threading

import numpy as np
import pytest

import cs_synth as S
import oracle
from _parity import compare

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cs(cuda_device):
    import paper_2609_35619_b300 as cs
    return cs


@pytest.fixture(scope="module")
def scenes(cs):
    a = S.apartment_scene(n=300_000, n_clusters=20)
    b = S.drone_scene(n=200_000)
    return [a, b], [cs.Scene(s["means"], s["scales"], s["quats"], s["opacity"]) for s in (a, b)]


def _alone(cs, scene, prims, ns, prim_type, G):
    params = cs.QueryParams(group_size=G)
    out = scene.query(torch.as_tensor(prims), ns, prim_type=prim_type, params=params, want_count=True)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _requests(n, seed):
    reqs = S.serving_requests(seed=seed, count=n, q_lo=1, q_hi=40_000)
    rng = np.random.default_rng(seed)
    for k, r in enumerate(reqs):
        r["G"] = int(rng.choice([0, 0, 1, 7, 32]))
        r["prim_type"] = 0
        if k % 5 == 3:  # some ellipsoid requests in the mix
            c = r["spheres"][:, :3].astype(np.float64)
            r["prims"] = S.ellipsoid_queries(seed + k, c).astype(np.float32)
            r["prim_type"] = 1
        else:
            r["prims"] = r["spheres"]
    return reqs


@pytest.mark.parametrize("use_graphs", [True, False])
def test_results_equal_alone_and_in_the_mix(cs, scenes, use_graphs):
    """With graph replay (the default: rows padded to the graph's bucket with
    primitives far outside the scenes) and with the kernels launched one by
    one."""
    data, sc = scenes
    reqs = _requests(120, 31)
    srv = cs.Server(sc, slots=2, slot_rows=1 << 17, max_requests=64, tile_config=0, use_graphs=use_graphs)
    tickets = [None] * len(reqs)

    def client(part):
        for k in range(part, len(reqs), 4):
            r = reqs[k]
            tickets[k] = srv.submit(r["scene"], r["prims"], r["nsigma"], prim_type=r["prim_type"],
                                    group_size=r["G"], want_count=True)

    th = [threading.Thread(target=client, args=(i,)) for i in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    results = [srv.wait(t, timeout=120.0) for t in tickets]
    st = srv.stats()
    srv.close()
    assert st["requests"] == len(reqs) and st["batches"] < len(reqs) and st["max_batch_requests"] > 1
    shared = sum(1 for _, tm in results if tm["batch_requests"] > 1)
    assert shared > len(reqs) // 4, shared
    for k, (r, (out, tm)) in enumerate(zip(reqs, results)):
        assert tm["submitted"] <= tm["launched"] <= tm["completed"]
        ref = _alone(cs, sc[r["scene"]], r["prims"], r["nsigma"], r["prim_type"], r["G"])
        for key in ("metric", "collide", "count"):
            np.testing.assert_array_equal(out[key], ref[key], err_msg=f"request {k} {key}")
        if r["G"] > 0:
            np.testing.assert_array_equal(out["group_metric"], ref["group_metric"], err_msg=f"request {k}")
            np.testing.assert_array_equal(out["group_collide"], ref["group_collide"], err_msg=f"request {k}")
    # a sample of rows against the oracle
    rng = np.random.default_rng(4)
    for k in rng.choice(len(reqs), 6, replace=False):
        r, out = reqs[k], results[k][0]
        rows = rng.choice(r["prims"].shape[0], min(64, r["prims"].shape[0]), replace=False)
        orc = oracle.query(data[r["scene"]], r["prims"][rows], r["prim_type"], r["nsigma"])
        compare({key: out[key][rows] for key in ("metric", "collide", "count")}, orc, 0, oracle.Params(),
                f"served request {k}")


def test_submit_validates_on_the_host(cs, scenes):
    _, sc = scenes
    srv = cs.Server(sc, slots=1, slot_rows=1024)
    good = np.array([[0.5, 0.5, 0.5, 0.1]], np.float32)
    bad = good.copy()
    bad[0, 1] = np.nan
    with pytest.raises(cs.CsError):
        srv.submit(0, bad, 1.0)
    with pytest.raises(cs.CsError):
        srv.submit(0, np.tile(good, (1025, 1)), 1.0)  # larger than a slot
    with pytest.raises(cs.CsError):
        srv.submit(2, good, 1.0)  # no such scene
    with pytest.raises(cs.CsError):
        srv.submit(0, good, -1.0)
    t = srv.submit(1, good, 1.0)
    out, tm = srv.wait(t, timeout=60.0)
    assert tm["batch_rows"] == 1 and out["metric"].shape == (1,)
    assert cs.abi.cs_server_wait(srv._h, t, 0.0, None) == cs.abi.CS_ERR_INVALID_ARG  # retired ticket
    srv.close()


def test_tuned_server_matches_plain_calls(cs, scenes):
    """A server whose tile shape comes from the autotuner gives the same bits."""
    _, sc = scenes
    reqs = _requests(24, 77)
    big = np.concatenate([r["spheres"] for r in reqs])
    sc[0].autotune(torch.as_tensor(big, device="cuda"), 1.0, reps=1)
    srv = cs.Server(sc[:1], slots=3, slot_rows=1 << 17)
    ts = [srv.submit(0, r["spheres"], r["nsigma"]) for r in reqs]
    res = [srv.wait(t, timeout=120.0)[0] for t in ts]
    srv.close()
    for r, out in zip(reqs, res):
        ref = _alone(cs, sc[0], r["spheres"], r["nsigma"], 0, 0)
        np.testing.assert_array_equal(out["metric"], ref["metric"])
        np.testing.assert_array_equal(out["collide"], ref["collide"])
