"""Derived ensemble quantities from per-cell ia_stats records (host post-processing).

Complex-formation probabilities with binomial (Wilson score) intervals (Fig. 3 and Fig. 4 of the
paper), mean ion heating with its standard error, the bounce-count histogram (Fig. 1c) and the
survival curve of complex lifetimes (Fig. 2: fraction of complexes alive after a time t).
"""
from __future__ import annotations

import math

import numpy as np

AU_TIME_S = 2.4188843265857e-17


def wilson(k: int, n: int, z: float = 3.0):
    """Wilson score interval of a binomial proportion at z standard deviations."""
    if n == 0:
        return 0.0, 0.0, 1.0
    p = k / n
    den = 1.0 + z * z / n
    mid = (p + z * z / (2 * n)) / den
    half = z * math.sqrt(p * (1 - p) / n + z * z / (4 * n * n)) / den
    return p, max(0.0, mid - half), min(1.0, mid + half)


def lifetime_edges_au(nbins: int = 64) -> np.ndarray:
    """Lower edges of the lifetime bins in a.u. of time: 2^(20 + k/2)."""
    return 2.0 ** (20.0 + 0.5 * np.arange(nbins + 1))


def summarize(rec) -> dict:
    """Derived quantities of one ia_stats record (a row of binding.STATS_DTYPE)."""
    n = int(rec["n"])
    k = int(rec["n_complex"])
    p, lo, hi = wilson(k, n)
    mean = float(rec["sum_dE"]) / n if n else 0.0
    var = max(float(rec["sum_dE2"]) / n - mean * mean, 0.0) if n else 0.0
    sem = math.sqrt(var / n) if n else 0.0
    lh = np.asarray(rec["lifetime_hist"], dtype=np.float64)
    alive = (lh[::-1].cumsum()[::-1] / lh.sum()) if lh.sum() > 0 else np.zeros_like(lh)
    edges = lifetime_edges_au(len(lh))
    return {
        "n": n, "P_complex": p, "P_complex_3sigma": (lo, hi),
        "mean_dE_ion": mean, "sem_dE_ion": sem,
        "bounce_hist": np.asarray(rec["bounce_hist"]).copy(),
        "survival_t_us": edges[:-1] * AU_TIME_S * 1e6, "survival": alive,
        "attempts_per_trajectory": float(rec["attempts"]) / n if n else 0.0,
    }
