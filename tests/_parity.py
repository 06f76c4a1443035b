"""Comparison of the CUDA path's outputs with the FP64 oracle, with the
tolerances of the parity contract:

  metric (mean/sum cost)  |gpu - oracle| <= 1e-5 |oracle|  (exact 0 for an
                          empty neighbour set)
  min / softmin st^2      the same, plus 8 u * cond for the FP32 rounding of
                          s^2 + n sqrt(sigma^2) when Eq. 8 cancels (u = 2^-24)
  counts                  exact
  collision flag          exact
Queries with a pair inside the cutoff band (|st^2 - S_cut| <= 1e-5 S_cut)
may change neighbour-set membership in FP32 and are excluded from the
metric/count checks; queries with a pair inside the collision band
(|st^2 - 1| <= 1e-5) are excluded from the flag/in-count checks; queries
whose Eq. 8 terms cancel strongly (cond = max over N_j of s^2 + n sqrt(sigma^2)
above 50, or cond_strict) are held to the derived bound 1e-5 + 16 u gamma cond
instead.  Every exclusion is counted and returned.

Thin ellipsoids: evaluating s^2 = d^T (A d) in FP32 with A = R P R^T rounds with
an error up to 8 u d^T|A|d <= 24 u kappa s^2, kappa = (a_max / a_min)^2 the
condition number of A, so a caller passing kappa per row gets the bound
24 u kappa cond (times gamma |metric| for the cost modes) added, and should
widen the oracle's bands by the same amount (oracle.Params.band).
"""
import numpy as np

U32 = 2.0 ** -24
REL = 1e-5
COND_STRICT = 50.0


def compare(gpu: dict, orc: dict, mode: int, params, label: str = "", check_count=True, kappa=None,
            cond_strict=COND_STRICT):
    import oracle
    metric_o = oracle.metric(orc, mode)
    g_metric = gpu["metric"].astype(np.float64)
    Q = metric_o.shape[0]
    band_cut = orc["band_cut"] > 0
    band_in = orc["band_in"] > 0
    strong = orc["cond"] > cond_strict
    report = {"Q": Q, "band_cut": int(band_cut.sum()), "band_in": int(band_in.sum()),
              "cancel": int((strong & ~band_cut).sum())}
    ok = ~band_cut
    # empty neighbour sets
    empty = (orc["count_nbr"] == 0) & ok
    if mode in (oracle.MODE_MEAN, oracle.MODE_SUM):
        assert np.all(g_metric[empty] == 0.0), f"{label}: empty sets must give exactly 0"
    else:
        assert np.all(np.isinf(g_metric[empty])), f"{label}: empty sets must give +inf"
    live = ok & ~empty
    o = metric_o[live]
    g = g_metric[live]
    if mode in (oracle.MODE_MEAN, oracle.MODE_SUM):
        tol = REL * np.abs(o) + np.where(strong[live], 16 * U32 * params.gamma * orc["cond"][live] * np.abs(o), 0.0)
    elif mode == oracle.MODE_MIN:
        tol = REL * np.abs(o) + 8 * U32 * orc["min_cond"][live] + 1e-30
    else:
        tol = REL * np.abs(o) + 8 * U32 * orc["cond"][live] + 1e-30
    if kappa is not None:
        kap = np.asarray(kappa, np.float64)[live]
        if mode in (oracle.MODE_MEAN, oracle.MODE_SUM):
            tol = tol + 24 * U32 * kap * params.gamma * orc["cond"][live] * np.abs(o)
        elif mode == oracle.MODE_MIN:
            tol = tol + 24 * U32 * kap * orc["min_cond"][live]
        else:
            tol = tol + 24 * U32 * kap * orc["cond"][live]
    err = np.abs(g - o)
    bad = err > tol
    assert not bad.any(), (
        f"{label}: {bad.sum()}/{live.sum()} metric mismatches; worst rel "
        f"{(err / np.maximum(np.abs(o), 1e-30)).max():.3e}; first: gpu={g[bad][:4]} oracle={o[bad][:4]}")
    if check_count and "count" in gpu:
        cnt_ok = gpu["count"][ok] == orc["count_nbr"][ok]
        assert cnt_ok.all(), f"{label}: {(~cnt_ok).sum()} neighbour-count mismatches"
    fl = ~band_in & ~band_cut
    col_ok = gpu["collide"][fl] == orc["collide"][fl]
    assert col_ok.all(), f"{label}: {(~col_ok).sum()} collision-flag mismatches"
    report["checked"] = int(live.sum())
    report["max_rel"] = float((err / np.maximum(np.abs(o), 1e-30)).max()) if live.any() else 0.0
    return report


def to_np(out: dict) -> dict:
    return {k: v.detach().cpu().numpy() for k, v in out.items()}
