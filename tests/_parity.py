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
(|st^2 - 1| <= 1e-5) are excluded from the flag/in-count checks; cost-mode
queries whose Eq. 8 terms cancel strongly are held to the derived bound
1e-5 + 16 u gamma cond_cost instead: the FP32 error of st^2 is at most about
8 u (s^2 + n sqrt(sigma^2)), and Eq. 11 turns an error e of st^2 into a
relative error gamma e of the pair's cost, except below s_min, where the cost
is flat (exactly d_max on both sides); cond_cost is the oracle's largest
s^2 + n sqrt(sigma^2) over the neighbours at or above s_min, and "strongly"
means above 50 (or cond_strict).  Every exclusion is counted and returned,
and the rows under the widened bound may be at most `max_cancel` of the rows
(5 % by default; at the default threshold every workload the tests use stays
below 1.5 %, measured with the oracle at n_sigma 2).

Thin ellipsoids: evaluating s^2 = d^T (A d) in FP32 with A = R P R^T rounds with
an error up to 8 u d^T|A|d <= 24 u kappa s^2, kappa = (a_max / a_min)^2 the
condition number of A, so a caller passing kappa per row gets the bound
24 u kappa cond (times gamma |metric| for the cost modes) added, and should
widen the oracle's bands by the same amount (oracle.Params.band).

Group outputs (Section II-D sums over links and horizon, Section II-E OR over
an edge) are checked by compare_groups, whose bound is derived below.
"""
import math

import numpy as np

U32 = 2.0 ** -24
REL = 1e-5
COND_STRICT = 50.0
MAX_CANCEL = 0.05
GROUP_WARP_MIN = 32  # groups of at least this many rows are summed by one warp


def compare(gpu: dict, orc: dict, mode: int, params, label: str = "", check_count=True, kappa=None,
            cond_strict=COND_STRICT, max_cancel=MAX_CANCEL):
    import oracle
    metric_o = oracle.metric(orc, mode)
    g_metric = gpu["metric"].astype(np.float64)
    Q = metric_o.shape[0]
    band_cut = orc["band_cut"] > 0
    band_in = orc["band_in"] > 0
    cost = mode in (oracle.MODE_MEAN, oracle.MODE_SUM)
    ccost = orc["cond_cost"]
    strong = (ccost > cond_strict) if cost else np.zeros(Q, bool)  # rows whose bound is widened
    report = {"Q": Q, "band_cut": int(band_cut.sum()), "band_in": int(band_in.sum()),
              "cancel": int((strong & ~band_cut).sum())}
    print(f"[parity] {label}: {report['cancel']}/{Q} rows under the cancellation bound (cond > {cond_strict:g}), "
          f"{report['band_cut']} in the cutoff band, {report['band_in']} in the collision band")
    assert report["cancel"] <= max(1, max_cancel * Q), (
        f"{label}: {report['cancel']}/{Q} rows take the widened cancellation bound (cap {max_cancel:.0%})")
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
    if cost:
        tol = REL * np.abs(o) + np.where(strong[live], 16 * U32 * params.gamma * ccost[live] * np.abs(o), 0.0)
    elif mode == oracle.MODE_MIN:
        tol = REL * np.abs(o) + 8 * U32 * orc["min_cond"][live] + 1e-30
    else:
        tol = REL * np.abs(o) + 8 * U32 * orc["cond"][live] + 1e-30
    if kappa is not None:
        kap = np.asarray(kappa, np.float64)[live]
        if cost:
            tol = tol + 24 * U32 * kap * params.gamma * ccost[live] * np.abs(o)
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
    # per-row bound for the group check (rows in the cutoff band: +inf; empty rows: exactly 0)
    row_tol = np.full(Q, np.inf)
    row_tol[empty] = 0.0
    row_tol[live] = tol
    report["row_tol"] = row_tol
    # relative widening of each row's bound for the cancellation of Eq. 8 (cost modes)
    report["cancel_rel"] = np.where(strong, 16 * U32 * params.gamma * ccost, 0.0)
    return report


def summation_depth(n: int, G: int) -> int:
    """Roundings on the longest path of the group sum of n rows in a launch
    with group size G: a warp (G >= 32) has each lane add ceil(n/32) rows in
    order (the first addition to 0 is exact), then a five-level shuffle tree;
    smaller groups are added in order by one thread."""
    if G >= GROUP_WARP_MIN:
        return (math.ceil(n / 32) - 1) + 5
    return max(n - 1, 0)


def cutoff_interval(sc, prims, prim_type: int, nsigma, params, rows, mode: int):
    """Oracle metrics of `rows` with the neighbour cutoff moved to
    S_cut (1 - band) and S_cut (1 + band): the pairs inside the cutoff band are
    all left out, or all taken in.  Each band pair has st^2 within band S_cut
    of S_cut, hence Eq. 11 cost e^{-gamma (S_cut - s_min)} d_max = eps d_max
    to within a factor e^{gamma band S_cut}: no neighbour costs less, so the
    mean cost falls (and the summed cost rises) with every band pair taken in,
    and any membership the FP32 path decides lies between the two, up to the
    spread of the band pairs' costs, eps d_max (e^{gamma band S_cut} -
    e^{-gamma band S_cut}), by which the interval is widened.  Returns
    (lo, hi) per row of `rows`."""
    import oracle
    out = []
    S = params.s_cut
    for f in (1.0 - params.band, 1.0 + params.band):
        eps = math.exp(-params.gamma * (S * f - params.s_min))
        p = oracle.Params(**{**params.__dict__, "eps": eps})
        o = oracle.query(sc, prims[rows], prim_type, nsigma if np.ndim(nsigma) == 0 else nsigma[rows], p)
        out.append(oracle.metric(o, mode))
    x = params.gamma * params.band * S
    spread = params.eps * params.d_max * (math.exp(x) - math.exp(-x))
    return np.minimum(out[0], out[1]) - spread, np.maximum(out[0], out[1]) + spread


def compare_groups(gpu_group_metric, gpu_group_collide, gpu_row_metric, orc: dict, rep: dict, G: int, mode: int,
                   label: str = "", interval=None):
    """Group outputs of one launch against the oracle's rows of whole groups.

    gpu_row_metric and orc cover whole groups (rows g G .. g G + G - 1 of each
    checked group, in order); rep is compare()'s report on those rows.  Bound
    for a group of n rows, with g_j the FP32 row metrics and o_j the oracle's:
        |fl(sum g_j) - sum o_j| <= sum_j |g_j - o_j| + gamma_m sum_j |g_j|,
    the first term bounded row by row by compare()'s tolerances, the second
    the rounding of the FP32 sum (m = summation_depth(n, G),
    gamma_m = m u / (1 - m u)).  A row in the cutoff band has no single oracle
    value: `interval` = (rows, lo, hi) from cutoff_interval gives the range its
    FP32 value may take, with the row tolerance applied to that range.  The
    group flag is an OR: it must be set when a row outside the collision band
    collides, and clear when no row can collide; otherwise it is not checked.
    Returns the number of groups checked."""
    import oracle
    o_rows = oracle.metric(orc, mode).astype(np.float64)
    g_rows = np.asarray(gpu_row_metric, np.float64)
    n_rows = o_rows.shape[0]
    lo = o_rows.copy()
    hi = o_rows.copy()
    tol = rep["row_tol"].copy()
    if interval is not None:
        rows, ilo, ihi = interval
        lo[rows] = np.minimum(lo[rows], ilo)
        hi[rows] = np.maximum(hi[rows], ihi)
        tol[rows] = (REL + rep["cancel_rel"][rows]) * np.maximum(np.abs(ilo), np.abs(ihi))
    assert np.isfinite(tol).all(), f"{label}: a row in the cutoff band has no interval"
    ng = (n_rows + G - 1) // G
    checked = 0
    for k in range(ng):
        b, e = k * G, min(n_rows, (k + 1) * G)
        n = e - b
        m = summation_depth(n, G)
        gam = m * U32 / (1 - m * U32)
        bound = tol[b:e].sum() + gam * np.abs(g_rows[b:e]).sum() + 1e-30
        got = float(gpu_group_metric[k])
        dist = max(lo[b:e].sum() - got, got - hi[b:e].sum(), 0.0)
        assert dist <= bound, (f"{label}: group {k}: gpu {got!r} outside [{lo[b:e].sum()!r}, {hi[b:e].sum()!r}] "
                               f"by {dist:.3e} > {bound:.3e}")
        certain = orc["band_in"][b:e] == 0
        hit = (orc["collide"][b:e] != 0) & certain
        if hit.any():
            assert gpu_group_collide[k] == 1, f"{label}: group {k} must collide"
        elif certain.all():
            assert gpu_group_collide[k] == 0, f"{label}: group {k} must be free"
        checked += 1
    return checked


def to_np(out: dict) -> dict:
    return {k: v.detach().cpu().numpy() for k, v in out.items()}
