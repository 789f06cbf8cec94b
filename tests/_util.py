"""Helpers shared by the tests (no method arithmetic here)."""
import numpy as np

TOL = 1e-4          # absolute tolerance on float32 values (rgb, unc, score, gamma/|P|, V)
GAP = 2e-4          # argmax must agree when the oracle's top-2 gap exceeds this


def sorted_gap(scores):
    s = np.sort(np.asarray(scores))
    return float(s[-1] - s[-2]) if len(s) > 1 else np.inf


def compare_views(gpu_unc, gpu_rgb, ref, tol=TOL):
    """Per-pixel comparison on pixels whose transmittance tests are not
    within the float32 rounding margin of eps_T.  Returns (max_err, n_amb)."""
    worst, n_amb = 0.0, 0
    for v in range(len(ref["unc"])):
        m = ~ref["amb"][v]
        n_amb += int((~m).sum())
        e = np.abs(gpu_unc[v][m] - ref["unc"][v][m]).max(initial=0.0)
        worst = max(worst, float(e))
        if gpu_rgb is not None:
            er = np.abs(gpu_rgb[v][:, m] - ref["rgb"][v][:, m]).max(initial=0.0)
            worst = max(worst, float(er))
    return worst, n_amb
