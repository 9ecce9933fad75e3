"""Derived ensemble quantities from per-cell ia_stats records (host post-processing).

Complex-formation probabilities with binomial (Wilson score) intervals (Fig. 3 and Fig. 4 of the
paper), mean ion heating with its standard error, the bounce-count histogram (Fig. 1c) and the
survival curve of complex lifetimes (Fig. 2: fraction of complexes alive after a time t) with
maximum-likelihood fits of its tail, and for Fig. 4 the heating energy scale W0^3D and a fit of the
complex probability's threshold energy.
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


# ------------------------------------------------------------------ Fig. 2: the lifetime tail

def lifetime_tail_fit(tau, t_min: float, t_cens: float | None = None, censored=None) -> dict:
    """Maximum-likelihood fits of the tail of complex lifetimes tau >= t_min (Fig. 2 discussion:
    beyond about 20 us the fraction of complexes alive decays as a power law, which marks
    non-hyperbolic chaos; hyperbolic chaos would decay exponentially).

    - Power law: the survival is S(t) = (t / t_min)^-gamma. Its estimator is
      gamma = d / sum ln(min(tau, t_cens) / t_min), the Hill estimator with right censoring.
    - Exponential: S(t) = exp(-lambda (t - t_min)), with lambda = d / sum (min(tau, t_cens) - t_min).

    d is the number of uncensored lifetimes. Censored lifetimes are lower bounds: complexes still alive
    when the run stopped. They are those at or beyond a common t_cens, or those flagged in `censored`
    (one flag per lifetime, for runs whose complexes started at different times before t_max).
    Returns both fits, their log-likelihoods and the standard error gamma / sqrt(d).
    """
    tau = np.asarray(tau, dtype=np.float64)
    flag = np.zeros(tau.shape, dtype=bool) if censored is None else np.asarray(censored, dtype=bool)
    keep = tau >= t_min
    tau, flag = tau[keep], flag[keep]
    if t_cens is None:
        t_cens = math.inf
    cens = (tau >= t_cens) | flag
    x = np.minimum(tau, t_cens)
    d = int((~cens).sum())
    n = int(tau.size)
    if d == 0:
        return {"n": n, "uncensored": 0, "gamma": math.nan, "gamma_se": math.nan, "rate": math.nan,
                "loglik_power": math.nan, "loglik_exp": math.nan}
    slog = float(np.log(x / t_min).sum())
    sexc = float((x - t_min).sum())
    gamma = d / slog
    rate = d / sexc
    # log-likelihoods of the uncensored densities and the censored survivals
    ll_pow = d * math.log(gamma / t_min) - (gamma + 1.0) * float(np.log(x[~cens] / t_min).sum()) \
        - gamma * float(np.log(x[cens] / t_min).sum())
    ll_exp = d * math.log(rate) - rate * sexc
    return {"n": n, "uncensored": d, "gamma": gamma, "gamma_se": gamma / math.sqrt(d), "rate": rate,
            "loglik_power": ll_pow, "loglik_exp": ll_exp}


def lifetime_tail_fit_binned(hist, k_min: int, ratio: float = math.sqrt(2.0)) -> dict:
    """Power-law exponent from a histogram of lifetimes over geometric bins (edges t_k = t_0 ratio^k,
    the ia_stats lifetime bins). Under S(t) ~ t^-gamma the bin index counted from k_min, j = K - k_min,
    is geometric: P(j) = (1 - p) p^j, where p = ratio^-gamma is the chance of reaching the next bin.
    The maximum-likelihood p is sum j / (d + sum j), d the uncensored count; the last bin, which also
    holds everything beyond it, is censored. Returns gamma = -ln p / ln ratio and its error from the
    Fisher information d / (p (1 - p)^2) by the delta method."""
    h = np.asarray(hist, dtype=np.float64)[k_min:]
    if h.sum() == 0:
        return {"n": 0, "gamma": math.nan, "gamma_se": math.nan}
    j = np.arange(h.size, dtype=np.float64)
    d = float(h[:-1].sum())
    s = float((j * h).sum())
    p = s / (d + s)
    gamma = -math.log(p) / math.log(ratio)
    se = math.sqrt(p * (1.0 - p) ** 2 / max(d, 1.0)) / p / math.log(ratio) if 0 < p < 1 else math.nan
    return {"n": int(h.sum()), "uncensored": int(d), "gamma": gamma, "gamma_se": se}


# ------------------------------------------------------------------ Fig. 4: the energy threshold

def w0_3d(m_atom: float, m_ion: float, Omega: float, a_x: float, q_x: float, C4: float) -> float:
    """Heating energy scale of a sympathetically cooled rf-trapped ion (Cetina, Grier & Vuletic 2012),
    as the paper writes it in the discussion of Fig. 4:
    W0 = 8 / (3 pi) (m_a / (m_i + m_a))^(5/3) (m_i^2 omega^4 C4 / q_x^2)^(1/3),
    omega = (Omega / 2) sqrt(a_x + q_x^2 / 2). Atomic units in, hartree out."""
    omega = 0.5 * Omega * math.sqrt(a_x + 0.5 * q_x * q_x)
    mass = (m_atom / (m_ion + m_atom)) ** (5.0 / 3.0)
    return 8.0 / (3.0 * math.pi) * mass * (m_ion ** 2 * omega ** 4 * C4 / (q_x * q_x)) ** (1.0 / 3.0)


def fit_threshold(E, k, n) -> dict:
    """Fit P(E) = P_inf + (P0 - P_inf) (1 - tanh((ln E - ln E_th) / w)) / 2 to complex counts k out
    of n at energies E. This is the Fig. 4 trend: the complex probability falls like a negative tanh
    up to a threshold energy. P_inf is what remains above the threshold; the paper's curves fall to
    zero.

    The fit is weighted least squares with the binomial variances (floored at 1/n). For each
    (ln E_th, w) on a grid, the two amplitudes enter linearly and are solved exactly. The best grid
    cell is refined three times. Returns:
      - E_th, the midpoint of the fall, in the units of E;
      - E_end = E_th e^w, where the fall has covered 88 % of P0 - P_inf (tanh 1 = 0.76);
      - w, P0, P_inf and chi2.
    """
    lnE = np.log(np.asarray(E, dtype=np.float64))
    k = np.asarray(k, dtype=np.float64)
    n = np.asarray(n, dtype=np.float64)
    f = k / n
    wt = n / np.maximum(f * (1.0 - f), 1.0 / n)

    def solve(ln_th, width):
        sh = 0.5 * (1.0 - np.tanh((lnE - ln_th) / width))
        A = np.stack([1.0 - sh, sh], axis=1)  # columns: P_inf, P0
        Aw = A * wt[:, None]
        coef = np.linalg.lstsq(Aw.T @ A, Aw.T @ f, rcond=None)[0]
        coef = np.clip(coef, 0.0, 1.0)
        r = f - A @ coef
        return float((wt * r * r).sum()), coef

    lo, hi = float(lnE.min()), float(lnE.max())
    best = (math.inf, None)
    for ln_th in np.linspace(lo, hi, 81):
        for width in np.geomspace(0.05, hi - lo, 40):
            c2, coef = solve(ln_th, width)
            if c2 < best[0]:
                best = (c2, (ln_th, width, coef))
    ln_th, width, coef = best[1]
    step_t, step_w = (hi - lo) / 80.0, width * 0.2
    for _ in range(3):
        for t in np.linspace(ln_th - step_t, ln_th + step_t, 11):
            for w in np.linspace(max(0.02, width - step_w), width + step_w, 11):
                c2, cf = solve(t, w)
                if c2 < best[0]:
                    best = (c2, (t, w, cf))
        ln_th, width, coef = best[1]
        step_t, step_w = step_t / 5.0, step_w / 5.0
    return {"E_th": math.exp(ln_th), "E_end": math.exp(ln_th + width), "width_ln": width,
            "P0": float(coef[1]), "P_inf": float(coef[0]), "chi2": best[0], "dof": int(len(f) - 4)}
