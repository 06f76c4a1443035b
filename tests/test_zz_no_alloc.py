"""cs_query_noalloc: the query for callers that cannot allocate device memory
while they run (a controller with a hard period, where cudaMalloc may block
and synchronise the device; a program whose device memory belongs to another
allocator).  Its results must equal cs_query's bit for bit (the same kernels
in the same order on the same rows), through the C ABI, on calls in a row that
share its fixed scratch area, and no call may take device memory.  Covered:
spheres in the default mode with groups and per-row n_sigma, ellipsoids at
exactly CS_QUERY_NOALLOC_MAX_ROWS rows, and the flags mode with groups (where
the per-group early-exit words live in the shared area and must start at zero).
Collected last so that a stop-at-first-failure run has run everything else
first; passes alone in a fresh process too.
"""

import numpy as np
import pytest

import cs_synth as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

_SCENE = {}


def _scene(cs):
    if "gpu" not in _SCENE:
        sc = S.drone_scene(n=200_000)
        _SCENE["gpu"] = cs.Scene(sc["means"], sc["scales"], sc["quats"], sc["opacity"])
    return _SCENE["gpu"]


def _outputs(Q, G, dev):
    ng = (Q + G - 1) // G
    # sentinel contents: outputs a mode does not write must keep them
    return {"metric": torch.full((Q,), -7.0, device=dev),
            "collide": torch.full((Q,), 9, dtype=torch.uint8, device=dev),
            "count": torch.full((Q,), -3, dtype=torch.int32, device=dev),
            "gm": torch.full((ng,), -5.0, device=dev),
            "gc": torch.full((ng,), 9, dtype=torch.uint8, device=dev)}


def _call(cs, fn, scene, prim_type, prims, ns, out, G, nsq=None, mode=None):
    kw = {"group_size": G}
    if mode is not None:
        kw["mode"] = mode
    p = cs.QueryParams(**kw).to_c()
    p.out_count = out["count"].data_ptr()
    p.out_group_metric = out["gm"].data_ptr()
    p.out_group_collide = out["gc"].data_ptr()
    if nsq is not None:
        p.nsigma_per_query = nsq.data_ptr()
    return fn(scene.handle, prim_type, prims, prims.shape[0], ns, out["metric"], out["collide"], p)


def _bits(t):
    a = t.cpu().numpy()
    return a.view(np.uint32) if a.dtype == np.float32 else a


def _same_bits(a, b):
    for k in ("metric", "collide", "count", "gm", "gc"):
        np.testing.assert_array_equal(_bits(a[k]), _bits(b[k]), err_msg=k)


def test_noalloc_equals_cs_query_on_two_calls_in_a_row(cuda_device):
    import paper_2609_35619_b300 as cs
    dev = cuda_device
    scene = _scene(cs)
    q_all = torch.as_tensor(S.drone_queries(rollouts=2048, horizon=32), device=dev)  # 65,536 rows
    # first call: 60,000 rows in groups of 32 at n_sigma = 1
    q1 = q_all[:60_000].contiguous()
    # second call: a different, smaller batch with per-row n_sigma and groups of 7
    q2 = q_all[-9_999:].contiguous()
    nsq = torch.as_tensor(np.random.default_rng(5).uniform(0, 2, q2.shape[0]).astype(np.float32), device=dev)
    sph = cs.CS_PRIM_SPHERE

    ref1, ref2 = _outputs(q1.shape[0], 32, dev), _outputs(q2.shape[0], 7, dev)
    assert _call(cs, cs.abi.cs_query, scene, sph, q1, 1.0, ref1, 32) == cs.abi.CS_OK
    assert _call(cs, cs.abi.cs_query, scene, sph, q2, 0.0, ref2, 7, nsq) == cs.abi.CS_OK
    torch.cuda.synchronize()

    got1, got2 = _outputs(q1.shape[0], 32, dev), _outputs(q2.shape[0], 7, dev)
    assert _call(cs, cs.abi.cs_query_noalloc, scene, sph, q1, 1.0, got1, 32) == cs.abi.CS_OK, cs.abi.cs_last_error()
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    assert _call(cs, cs.abi.cs_query_noalloc, scene, sph, q2, 0.0, got2, 7, nsq) == cs.abi.CS_OK, \
        cs.abi.cs_last_error()
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before, "the second call changed the free device memory"

    _same_bits(got1, ref1)
    _same_bits(got2, ref2)
    assert int(got1["count"].sum()) > 0 and int(got2["count"].sum()) > 0


def test_noalloc_ellipsoids_at_the_row_limit(cuda_device):
    """Ellipsoids use three prepared records per row, the largest part of the
    area; Q = CS_QUERY_NOALLOC_MAX_ROWS fills it exactly."""
    import paper_2609_35619_b300 as cs
    dev = cuda_device
    scene = _scene(cs)
    n = cs.abi.CS_QUERY_NOALLOC_MAX_ROWS
    centres = S.drone_queries(rollouts=n // 32, horizon=32)[:, :3]
    e = torch.as_tensor(S.ellipsoid_queries(77, centres, 0.03, 0.25), device=dev)
    assert e.shape[0] == n
    ell = cs.CS_PRIM_ELLIPSOID
    ref = _outputs(n, 64, dev)
    assert _call(cs, cs.abi.cs_query, scene, ell, e, 1.0, ref, 64) == cs.abi.CS_OK
    torch.cuda.synchronize()
    for _ in range(2):  # twice in a row on the same area
        got = _outputs(n, 64, dev)
        assert _call(cs, cs.abi.cs_query_noalloc, scene, ell, e, 1.0, got, 64) == cs.abi.CS_OK, \
            cs.abi.cs_last_error()
        torch.cuda.synchronize()
        _same_bits(got, ref)
    assert int(ref["count"].sum()) > 0 and int(ref["collide"].sum()) > 0


def test_noalloc_flags_mode_with_groups(cuda_device):
    """The flags mode writes only flags (metric, count and group metric keep
    the caller's contents), as cs_query does; group flags are exact and
    equal cs_query's; finished rows equal cs_query's flags; unfinished rows
    (2) only occur in colliding groups.  Run twice in a row, after a default
    call has left other contents in the area, so the group words must be
    cleared by the call itself."""
    import paper_2609_35619_b300 as cs
    dev = cuda_device
    scene = _scene(cs)
    q = torch.as_tensor(S.drone_queries(rollouts=2048, horizon=32, radius=0.3), device=dev)
    Q, G = q.shape[0], 32
    sph, FLAGS = cs.CS_PRIM_SPHERE, cs.CS_METRIC_FLAGS
    full = _outputs(Q, G, dev)  # the full evaluation's flags (default mode)
    assert _call(cs, cs.abi.cs_query, scene, sph, q, 1.0, full, G) == cs.abi.CS_OK
    ref = _outputs(Q, G, dev)
    assert _call(cs, cs.abi.cs_query, scene, sph, q, 1.0, ref, G, mode=FLAGS) == cs.abi.CS_OK
    torch.cuda.synchronize()
    gg = full["gc"].cpu().numpy()
    assert gg.sum() > 0 and (gg == 0).sum() > 0, "the batch must have colliding and free groups"
    for _ in range(2):
        got = _outputs(Q, G, dev)
        assert _call(cs, cs.abi.cs_query_noalloc, scene, sph, q, 1.0, got, G, mode=FLAGS) == cs.abi.CS_OK, \
            cs.abi.cs_last_error()
        torch.cuda.synchronize()
        for k, v in (("metric", -7.0), ("count", -3), ("gm", -5.0)):
            assert (got[k].cpu().numpy() == v).all(), f"flags mode wrote {k}"
        np.testing.assert_array_equal(got["gc"].cpu().numpy(), ref["gc"].cpu().numpy())
        np.testing.assert_array_equal(got["gc"].cpu().numpy(), gg)
        row, frow = got["collide"].cpu().numpy(), full["collide"].cpu().numpy()
        assert np.isin(row, (0, 1, 2)).all()
        done = row != 2
        np.testing.assert_array_equal(row[done], frow[done])
        assert (gg[np.flatnonzero(~done) // G] == 1).all(), "unfinished rows only in colliding groups"
        # a metric-only request in the flags mode asks for nothing that is computed
        p = cs.QueryParams(mode=FLAGS).to_c()
        st = cs.abi.cs_query_noalloc(scene.handle, sph, q, Q, 1.0, got["metric"], None, p)
        assert st == cs.abi.CS_ERR_INVALID_ARG


def test_noalloc_rejects_oversize_and_host_buffers(cuda_device):
    import paper_2609_35619_b300 as cs
    sc = S.tiny_scene()
    scene = cs.Scene(sc["means"], sc["scales"], sc["quats"], sc["opacity"])
    n = cs.abi.CS_QUERY_NOALLOC_MAX_ROWS + 1
    prims = torch.zeros((n, 4), device=cuda_device)
    prims[:, 3] = 0.1
    out = torch.empty(n, device=cuda_device)
    st = cs.abi.cs_query_noalloc(scene.handle, 0, prims, n, 1.0, out, None, None)
    assert st == cs.abi.CS_ERR_INVALID_ARG and "65536" in cs.abi.cs_last_error()
    p = cs.QueryParams().to_c()
    p.host_io = 1
    h = np.zeros((4, 4), np.float32)
    st = cs.abi.cs_query_noalloc(scene.handle, 0, h, 4, 1.0, np.zeros(4, np.float32), None, p)
    assert st == cs.abi.CS_ERR_INVALID_ARG
