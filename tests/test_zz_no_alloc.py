"""cs_query_noalloc: the query for callers that cannot allocate device memory
while they run (a controller with a hard period, where cudaMalloc may block
and synchronise the device; a program whose device memory belongs to another
allocator).  Its results must equal cs_query's, through the C ABI, on two
calls in a row that share its fixed scratch area, and neither call may take
device memory.  Collected last so that a stop-at-first-failure run has run
everything else first; passes alone in a fresh process too.
"""

import numpy as np
import pytest

import cs_synth as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

REL = 1e-5  # the parity tolerance of the metric


def _outputs(Q, G, dev):
    ng = (Q + G - 1) // G
    return {"metric": torch.empty(Q, device=dev), "collide": torch.empty(Q, dtype=torch.uint8, device=dev),
            "count": torch.empty(Q, dtype=torch.int32, device=dev),
            "gm": torch.empty(ng, device=dev), "gc": torch.empty(ng, dtype=torch.uint8, device=dev)}


def _call(cs, fn, scene, prims, ns, out, G, nsq=None):
    p = cs.QueryParams(group_size=G).to_c()
    p.out_count = out["count"].data_ptr()
    p.out_group_metric = out["gm"].data_ptr()
    p.out_group_collide = out["gc"].data_ptr()
    if nsq is not None:
        p.nsigma_per_query = nsq.data_ptr()
    return fn(scene.handle, cs.CS_PRIM_SPHERE, prims, prims.shape[0], ns, out["metric"], out["collide"], p)


def _same(a, b):
    m_a, m_b = a["metric"].cpu().numpy().astype(np.float64), b["metric"].cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(m_a, m_b, rtol=REL, atol=0)
    np.testing.assert_array_equal(a["collide"].cpu().numpy(), b["collide"].cpu().numpy())
    np.testing.assert_array_equal(a["count"].cpu().numpy(), b["count"].cpu().numpy())
    np.testing.assert_allclose(a["gm"].cpu().numpy(), b["gm"].cpu().numpy(), rtol=REL, atol=0)
    np.testing.assert_array_equal(a["gc"].cpu().numpy(), b["gc"].cpu().numpy())


def test_noalloc_equals_cs_query_on_two_calls_in_a_row(cuda_device):
    import paper_2609_35619_b300 as cs
    dev = cuda_device
    sc = S.drone_scene(n=200_000)
    scene = cs.Scene(sc["means"], sc["scales"], sc["quats"], sc["opacity"])
    q_all = torch.as_tensor(S.drone_queries(rollouts=2048, horizon=32), device=dev)  # 65,536 rows
    # first call: 60,000 rows in groups of 32 at n_sigma = 1
    q1 = q_all[:60_000].contiguous()
    # second call: a different, smaller batch with per-row n_sigma and groups of 7
    q2 = q_all[-9_999:].contiguous()
    nsq = torch.as_tensor(np.random.default_rng(5).uniform(0, 2, q2.shape[0]).astype(np.float32), device=dev)

    ref1, ref2 = _outputs(q1.shape[0], 32, dev), _outputs(q2.shape[0], 7, dev)
    assert _call(cs, cs.abi.cs_query, scene, q1, 1.0, ref1, 32) == cs.abi.CS_OK
    assert _call(cs, cs.abi.cs_query, scene, q2, 0.0, ref2, 7, nsq) == cs.abi.CS_OK
    torch.cuda.synchronize()

    got1, got2 = _outputs(q1.shape[0], 32, dev), _outputs(q2.shape[0], 7, dev)
    assert _call(cs, cs.abi.cs_query_noalloc, scene, q1, 1.0, got1, 32) == cs.abi.CS_OK, cs.abi.cs_last_error()
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    assert _call(cs, cs.abi.cs_query_noalloc, scene, q2, 0.0, got2, 7, nsq) == cs.abi.CS_OK, cs.abi.cs_last_error()
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before, "the second call changed the free device memory"

    _same(got1, ref1)
    _same(got2, ref2)
    assert int(got1["count"].sum()) > 0 and int(got2["count"].sum()) > 0


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
