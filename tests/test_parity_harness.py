"""The parity harness itself, on the CPU: the oracle's own rows rounded to
FP32 and summed in FP32 the way a warp sums a group must pass compare() and
compare_groups(); a group sum moved beyond the derived bound, a wrong group
flag, or too many rows under the cancellation bound must fail."""
import numpy as np
import pytest

import cs_synth as S
import oracle
from _parity import compare, compare_groups, cutoff_interval, summation_depth


def _warp_sum32(x):
    """FP32 group sum in the order of a warp: lane l adds rows l, l + 32, ...
    in order, then a shuffle tree (xor 16, 8, 4, 2, 1)."""
    lanes = np.zeros(32, np.float32)
    for j, v in enumerate(np.asarray(x, np.float32)):
        lanes[j % 32] = np.float32(lanes[j % 32] + v)
    for o in (16, 8, 4, 2, 1):
        lanes = (lanes + lanes[np.arange(32) ^ o]).astype(np.float32)
    return lanes[0]


def _fake_gpu(orc, G):
    m = orc["mean_cost"].astype(np.float32)
    Q = m.shape[0]
    ng = (Q + G - 1) // G
    if G >= 32:
        gm = np.array([_warp_sum32(m[k * G:(k + 1) * G]) for k in range(ng)], np.float32)
    else:
        gm = np.array([np.cumsum(m[k * G:(k + 1) * G], dtype=np.float32)[-1] for k in range(ng)], np.float32)
    gc = np.array([orc["collide"][k * G:(k + 1) * G].max() for k in range(ng)], np.uint8)
    return {"metric": m, "collide": orc["collide"].copy(), "count": orc["count_nbr"].astype(np.int32)}, gm, gc


@pytest.fixture(scope="module")
def tiny():
    sc = S.tiny_scene()
    q = S.tiny_queries(q=1000)
    P = oracle.Params()
    orc = oracle.query(sc, q, 0, 1.0, P)
    band = np.flatnonzero(orc["band_cut"] > 0)
    return sc, q, P, orc, band, cutoff_interval(sc, q, 0, 1.0, P, band, oracle.MODE_MEAN)


@pytest.mark.parametrize("G", [7, 32, 64, 1000])
def test_groups_of_fp32_rows_pass(tiny, G):
    sc, q, P, orc, band, (lo, hi) = tiny
    gpu, gm, gc = _fake_gpu(orc, G)
    rep = compare(gpu, orc, 0, P, "fp32 rows")
    n = compare_groups(gm, gc, gpu["metric"], orc, rep, G, oracle.MODE_MEAN, "fp32 groups", interval=(band, lo, hi))
    assert n == gm.shape[0]


def test_group_sum_beyond_the_bound_fails(tiny):
    sc, q, P, orc, band, (lo, hi) = tiny
    G = 64
    gpu, gm, gc = _fake_gpu(orc, G)
    rep = compare(gpu, orc, 0, P, "fp32 rows")
    k = 3
    b, e = k * G, (k + 1) * G
    bound = rep["row_tol"][b:e][np.isfinite(rep["row_tol"][b:e])].sum()
    m = summation_depth(G, G)
    bound += m * 2.0 ** -24 * np.abs(gpu["metric"][b:e]).sum() + np.abs(hi - lo).sum()
    bad = gm.copy()
    bad[k] = np.float32(orc["mean_cost"][b:e].sum() + 4 * bound)
    with pytest.raises(AssertionError, match="outside"):
        compare_groups(bad, gc, gpu["metric"], orc, rep, G, oracle.MODE_MEAN, "moved", interval=(band, lo, hi))
    flip = gc.copy()
    certain = np.array([(orc["band_in"][j * G:(j + 1) * G] == 0).all() for j in range(gc.shape[0])])
    j = int(np.flatnonzero(certain)[0])
    flip[j] ^= 1
    with pytest.raises(AssertionError, match="must"):
        compare_groups(gm, flip, gpu["metric"], orc, rep, G, oracle.MODE_MEAN, "flag", interval=(band, lo, hi))


def test_band_rows_need_an_interval(tiny):
    sc, q, P, orc, band, _ = tiny
    assert band.size > 0, "the tiny batch has rows in the cutoff band"
    gpu, gm, gc = _fake_gpu(orc, 64)
    rep = compare(gpu, orc, 0, P, "fp32 rows")
    with pytest.raises(AssertionError, match="no interval"):
        compare_groups(gm, gc, gpu["metric"], orc, rep, 64, oracle.MODE_MEAN, "no interval")


def test_cutoff_interval_brackets_the_memberships(tiny):
    """Each band row's oracle metric at the nominal cutoff lies in its
    interval, and the interval is no wider than taking in k near-zero
    members can move a mean of n: (S/n) k/(n + k) <= hi k/|N_j|."""
    sc, q, P, orc, band, (lo, hi) = tiny
    m = orc["mean_cost"][band]
    assert (lo <= m).all() and (m <= hi).all()
    k = orc["band_cut"][band]
    assert (hi - lo <= hi * k / orc["count_nbr"][band] + 1e-12).all()


def test_cancellation_cap(tiny):
    sc, q, P, orc, band, _ = tiny
    gpu, _, _ = _fake_gpu(orc, 64)
    forged = dict(orc, cond_cost=np.where(np.arange(orc["cond"].shape[0]) % 10 == 0, 100.0, orc["cond_cost"]))
    with pytest.raises(AssertionError, match="cancellation bound"):
        compare(gpu, forged, 0, P, "forged cond")
    rep = compare(gpu, forged, 0, P, "forged cond, cap raised", max_cancel=0.2)
    assert rep["cancel"] >= 90
