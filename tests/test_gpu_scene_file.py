"""Checkpoint and resume of a built scene (cs_scene_save / cs_scene_load):
a scene read back from its file answers every query bit for bit as the
scene that wrote it (same layout, same chunk order), its info and export
match, the appearance of the render path travels with it, and the loaded
scene still matches the FP64 oracle.  Loading validates the file before it
allocates."""
import ctypes

import numpy as np
import pytest

import cs_synth as S
import oracle
from _parity import compare, to_np

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cs(cuda_device):
    import paper_2609_35619_b300 as cs
    return cs


def _same(a, b, label, skip=()):
    assert a.keys() == b.keys(), label
    for k in a:
        if k in skip:
            continue
        x, y = a[k].cpu().numpy(), b[k].cpu().numpy()
        assert x.dtype == y.dtype and x.shape == y.shape, (label, k)
        assert np.array_equal(x.view(np.uint8), y.view(np.uint8)), f"{label}: {k} differs"


def _round_trip(cs, scene, tmp_path, name):
    path = tmp_path / name
    scene.save(path)
    assert path.stat().st_size > scene.info()["device_bytes"]
    return cs.Scene.load(path)


def test_tiny_scene_bit_exact_and_oracle(cs, tmp_path):
    sc = S.tiny_scene()
    q = S.tiny_queries(q=1000)
    a = cs.Scene(sc["means"], sc["scales"], sc["quats"], sc["opacity"])
    b = _round_trip(cs, a, tmp_path, "tiny.csscene")
    assert a.info() == b.info()
    for x, y in zip(a.export(), b.export()):
        assert torch.equal(x, y)
    qt = torch.as_tensor(q, device="cuda")
    runs = [
        dict(nsigma=1.0, want_count=True, params=cs.QueryParams(group_size=32)),
        dict(nsigma=0.0, want_count=True, params=cs.QueryParams(sweep=(0.0, 1.0, 2.0), tile_config=27)),
        dict(nsigma=2.0, params=cs.QueryParams(mode=cs.CS_METRIC_SOFTMIN_S2, tile_config=28)),
        dict(nsigma=1.0, params=cs.QueryParams(mode=cs.CS_METRIC_FLAGS)),
        dict(nsigma=1.0, params=cs.QueryParams(mode=cs.CS_METRIC_FLAGS, group_size=16)),
    ]
    for i, kw in enumerate(runs):
        # The flags mode writes only the collision outputs; with groups a row's
        # own flag may read "not finished" (2) depending on when its group was
        # settled, and only the group flag is exact.
        p = kw["params"]
        skip = ()
        if p.mode == cs.CS_METRIC_FLAGS:
            skip = ("metric", "group_metric") + (("collide",) if p.group_size else ())
        _same(a.query(qt, **kw), b.query(qt, **kw), f"run {i}", skip)
    assert torch.equal(a.query_grad(qt, 1.0), b.query_grad(qt, 1.0))
    e = torch.as_tensor(S.ellipsoid_queries(4, np.random.default_rng(3).uniform(0, 2, (500, 3))), device="cuda")
    _same(a.query(e, 1.0, prim_type=1, want_count=True), b.query(e, 1.0, prim_type=1, want_count=True), "ellipsoids")
    a.sync()
    b.sync()
    # the loaded scene on its own against the FP64 oracle
    P = oracle.Params()
    out = to_np(b.query(qt, 1.0, want_count=True))
    b.sync()
    compare(out, oracle.query(sc, q, 0, 1.0, P), 0, P, "loaded scene")
    # the original may go first: the loaded scene owns its own memory
    a.close()
    out2 = to_np(b.query(qt, 1.0, want_count=True))
    assert all(np.array_equal(out[k], out2[k], equal_nan=True) for k in out)


def test_multi_level_tree_and_appearance(cs, tmp_path):
    """200,000 Gaussians (three node levels, a large tier), with the render
    path's appearance set: queries and images agree bit for bit."""
    sc = S.drone_scene(n=200_000)
    a = cs.Scene(sc["means"], sc["scales"], sc["quats"], sc["opacity"])
    a.set_appearance(sc["opacity"], S.scene_colors(sc))
    inf = a.info()
    assert inf["n_large"] > 0 and all(d >= 1 for d in inf["dims"]) and inf["dims"][0] > 32
    b = _round_trip(cs, a, tmp_path, "drone.csscene")
    assert b.info() == inf
    q = torch.as_tensor(S.drone_queries(rollouts=256, horizon=32).reshape(-1, 4), device="cuda")
    _same(a.query(q, 1.0, want_count=True), b.query(q, 1.0, want_count=True), "drone spheres")
    cams = np.stack([S.look_at([0.5 + i, 0.5, 1.2], [3.0, 3.0, 1.0], f=60, width=64, height=48) for i in range(3)])
    ct = torch.as_tensor(cams, device="cuda")
    _same(a.render(ct, 64, 48), b.render(ct, 64, 48), "render")
    a.sync()
    b.sync()


def test_empty_scene(cs, tmp_path):
    z = np.zeros((0, 3), np.float32)
    a = cs.Scene(z, z, np.zeros((0, 4), np.float32))
    b = _round_trip(cs, a, tmp_path, "empty.csscene")
    assert b.info()["n_kept"] == 0
    q = torch.as_tensor(S.tiny_queries(q=100), device="cuda")
    out = to_np(b.query(q, 1.0, want_count=True))
    b.sync()
    assert (out["count"] == 0).all() and (out["metric"] == 0).all() and (out["collide"] == 0).all()


def test_load_rejects_a_damaged_file(cs, tmp_path):
    sc = S.tiny_scene()
    a = cs.Scene(sc["means"], sc["scales"], sc["quats"], sc["opacity"])
    path = tmp_path / "ok.csscene"
    a.save(path)
    raw = bytearray(path.read_bytes())
    out = ctypes.c_void_p()
    bad = tmp_path / "bad.csscene"
    bad.write_bytes(bytes(raw[:-7]))  # truncated
    assert cs.abi.cs_scene_load(str(bad), None, out) == cs.abi.CS_ERR_INVALID_ARG and not out
    assert "truncated" in cs.abi.cs_last_error()
    hdr = 192
    slot_off = int(np.frombuffer(bytes(raw[184:192]), "<i8")[0])
    dmg = bytearray(raw)
    dmg[hdr + slot_off:hdr + slot_off + 4] = np.int32(1 << 30).tobytes()  # a slot index out of range
    bad.write_bytes(bytes(dmg))
    assert cs.abi.cs_scene_load(str(bad), None, out) == cs.abi.CS_ERR_INVALID_ARG and not out
    assert "slot index" in cs.abi.cs_last_error()
