"""Helpers shared by the tests (no method arithmetic here).

The oracle gives, for every output that a transmittance test near eps_T can
change, the least and greatest value that output takes over every place
where the run could stop when the tests inside the band
[eps_T (1 - m), eps_T (1 + m)] go either way (m = the oracle's margin).
A float32 pass whose transmittance stays within relative m of the float64
one stops inside that range, so its outputs must lie in [lo, hi] up to the
value tolerance; where no test falls in the band, lo = hi = the oracle's
value and the check is the plain element-by-element one.  Nothing is left
out of the comparison.
"""
import numpy as np

TOL = 1e-4          # absolute tolerance on float32 values (rgb, unc, score, gamma/|P|, V)
GAP = 2e-4          # argmax must agree when the oracle's top-2 gap exceeds this
EPS_T = 1e-4        # the default transmittance threshold
MARGIN = 1e-3       # the oracle's band around it (relative)


def sorted_gap(scores):
    s = np.sort(np.asarray(scores))
    return float(s[-1] - s[-2]) if len(s) > 1 else np.inf


def excess(x, lo, hi):
    """Distance of x outside [lo, hi] (0 inside), elementwise."""
    x = np.asarray(x, np.float64)
    return np.maximum(np.maximum(lo - x, x - hi), 0.0)


def compare_views(gpu_unc, gpu_rgb, ref, tol=TOL):
    """Largest distance of the GPU's per-pixel entropy and colour from the
    oracle's ranges, over every pixel of every view; and the number of pixels
    whose range is wider than a point (a transmittance test in the band)."""
    worst, n_band = 0.0, 0
    for v in range(len(ref["unc"])):
        b = ref["bnd"][v]
        n_band += int(((b["unc_hi"] > b["unc_lo"]) | (b["rgb_hi"] > b["rgb_lo"]).any(0)).sum())
        worst = max(worst, float(excess(gpu_unc[v], b["unc_lo"], b["unc_hi"]).max(initial=0.0)))
        if gpu_rgb is not None:
            worst = max(worst, float(excess(gpu_rgb[v], b["rgb_lo"], b["rgb_hi"]).max(initial=0.0)))
    return worst, n_band


def score_excess(gpu_score, ref):
    """Distance of each GPU view score from the oracle's range of scores."""
    return excess(gpu_score, ref["score_lo"], ref["score_hi"])


def visibility_check(sumT, cnt, bnd, eps=EPS_T, margin=MARGIN):
    """Per Gaussian of one view: the GPU's count must lie in the oracle's
    [early, late] count range (integers: exactly), and its mean
    transmittance v = sumT / cnt must lie in the range that count allows --
    the early entries' sum plus, for each of the cnt - cnt_early later
    entries, a transmittance in [eps (1 - m)^2, eps (1 + m)^2].
    Returns (count violations, largest v excess, number of Gaussians whose
    count differs from the early count)."""
    ce, cl, se = bnd["cnt_early"], bnd["cnt_late"], bnd["sum_early"]
    cnt = np.asarray(cnt, np.int64)
    bad_cnt = int(((cnt < ce) | (cnt > cl)).sum())
    k = np.clip(cnt - ce, 0, None).astype(np.float64)
    tlo, thi = eps * (1 - margin) ** 2, eps * (1 + margin) ** 2
    c1 = np.maximum(cnt, 1).astype(np.float64)
    v = np.where(cnt > 0, sumT / c1, 0.0)
    vlo = np.where(cnt > 0, (se + k * tlo) / c1, 0.0)
    vhi = np.where(cnt > 0, (se + k * thi) / c1, 0.0)
    return bad_cnt, float(excess(v, vlo, vhi).max(initial=0.0)), int((cnt != ce).sum())
