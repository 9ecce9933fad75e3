"""Host-side fits of the paper's ensemble figures (CPU only), pinned on synthetic samples drawn from
the laws they estimate.

- Fig. 2: the power-law tail of complex lifetimes, from per-trajectory lifetimes and from the
  geometric-bin histogram.
- Fig. 4: the threshold energy of the complex probability and the heating scale W0^3D.
"""
import math

import numpy as np
import pytest

from paper_2509_15117_gb300 import inputs as I
from paper_2509_15117_gb300 import statistics as St


def pareto(n, gamma, t_min, seed):
    u = np.random.default_rng(seed).random(n)
    return t_min * (1.0 - u) ** (-1.0 / gamma)


@pytest.mark.parametrize("gamma", [0.5, 1.3, 2.0])
def test_power_law_tail_recovered(gamma):
    tau = pareto(50_000, gamma, 20.0, seed=int(gamma * 10))
    f = St.lifetime_tail_fit(np.concatenate([tau, [1.0, 5.0]]), t_min=20.0)  # below t_min: ignored
    assert f["n"] == 50_000
    assert abs(f["gamma"] - gamma) < 4 * f["gamma_se"]
    assert f["loglik_power"] > f["loglik_exp"]


def test_censored_power_law_tail():
    gamma, t_min, t_c = 1.0, 20.0, 600.0
    tau = pareto(80_000, gamma, t_min, seed=3)
    f_cens = St.lifetime_tail_fit(np.minimum(tau, t_c), t_min, t_cens=t_c)
    assert f_cens["uncensored"] == int((tau < t_c).sum())
    assert abs(f_cens["gamma"] - gamma) < 4 * f_cens["gamma_se"]
    # ignoring the censoring biases the exponent upward, well beyond the error
    f_naive = St.lifetime_tail_fit(np.minimum(tau, t_c) * (1 - 1e-15), t_min)
    assert f_naive["gamma"] > gamma + 4 * f_naive["gamma_se"]


def test_power_law_tail_with_per_lifetime_censoring():
    """Complexes that start at different times and are all stopped at the same t_max: each lifetime
    is censored at its own bound, t_max - t_start."""
    rng = np.random.default_rng(9)
    gamma, t_min = 0.8, 20.0
    tau = pareto(80_000, gamma, t_min, seed=11)
    bound = rng.uniform(200.0, 1000.0, tau.size)
    cens = tau >= bound
    f = St.lifetime_tail_fit(np.minimum(tau, bound), t_min, censored=cens)
    assert f["uncensored"] == int((~cens).sum()) and cens.sum() > 1000
    assert abs(f["gamma"] - gamma) < 4 * f["gamma_se"]


def test_exponential_tail_is_told_apart():
    tau = 20.0 + np.random.default_rng(4).exponential(50.0, 50_000)
    f = St.lifetime_tail_fit(tau, 20.0)
    assert f["loglik_exp"] > f["loglik_power"]
    assert f["rate"] == pytest.approx(1 / 50.0, rel=0.03)


def test_binned_tail_on_the_lifetime_bins():
    """Pareto lifetimes put in the ia_stats bins (edges 2^(20 + k/2) a.u.): the binned estimator
    recovers the exponent; everything past the last bin lands in it (censored)."""
    edges = St.lifetime_edges_au(64)
    for gamma in (0.7, 1.5):
        tau = pareto(100_000, gamma, edges[10], seed=int(gamma * 100))
        k = np.clip(np.floor(2.0 * (np.log2(tau) - 20.0)).astype(int), 0, 63)
        hist = np.bincount(k, minlength=64)
        f = St.lifetime_tail_fit_binned(hist, 10)
        assert f["n"] == 100_000
        assert abs(f["gamma"] - gamma) < 4 * f["gamma_se"], (gamma, f)
        # a cut that truncates the tail at bin 24 still works: the censoring handles the last bin
        hist_cut = hist.copy()
        hist_cut[24] = hist[24:].sum()
        hist_cut[25:] = 0
        f2 = St.lifetime_tail_fit_binned(hist_cut[:25], 10)
        assert abs(f2["gamma"] - gamma) < 4 * f2["gamma_se"], (gamma, f2)


def test_w0_scaling_laws():
    """The paper: with Omega fixed and a_x << q_x^2/2, W0 scales as q_x^(2/3). The formula also
    scales as C4^(1/3), and as (m_a / (m_i + m_a))^(5/3) at fixed ion mass."""
    d = I.make_system("Rb")
    C4 = 0.5 * d.alpha
    w = St.w0_3d(d.m_atom, d.m_ion, d.Omega, 0.0, 0.1, C4)
    assert St.w0_3d(d.m_atom, d.m_ion, d.Omega, 0.0, 0.2, C4) / w == pytest.approx(2.0 ** (2.0 / 3.0), rel=1e-12)
    assert St.w0_3d(d.m_atom, d.m_ion, d.Omega, 0.0, 0.1, 8 * C4) / w == pytest.approx(2.0, rel=1e-12)
    m2 = 2 * d.m_atom
    ratio = ((m2 / (d.m_ion + m2)) / (d.m_atom / (d.m_ion + d.m_atom))) ** (5.0 / 3.0)
    assert St.w0_3d(m2, d.m_ion, d.Omega, 0.0, 0.1, C4) / w == pytest.approx(ratio, rel=1e-12)
    # a small static a_x raises omega: W0 grows with a_x > 0
    assert St.w0_3d(d.m_atom, d.m_ion, d.Omega, 1e-3, 0.1, C4) > w
    # order of magnitude: microkelvin for Yb+-Rb at q = 0.1, 2 MHz (the Fig. 4 energy axis)
    assert 1e-6 < w / I.K_TO_HARTREE < 1e-4


@pytest.mark.parametrize("p_inf", [0.0, 0.1])
def test_threshold_fit_recovers_a_negative_tanh(p_inf):
    rng = np.random.default_rng(5)
    E = np.geomspace(1e-7, 1e-3, 100)
    p0, th, width = 0.6, 3e-5, 0.8
    p = p_inf + (p0 - p_inf) * 0.5 * (1 - np.tanh((np.log(E) - math.log(th)) / width))
    n = np.full(100, 10_000)
    k = rng.binomial(n, p)
    f = St.fit_threshold(E, k, n)
    assert f["E_th"] == pytest.approx(th, rel=0.05)
    assert f["width_ln"] == pytest.approx(width, rel=0.05)
    assert f["P0"] == pytest.approx(p0, abs=0.01)
    assert f["P_inf"] == pytest.approx(p_inf, abs=0.005)
    assert f["chi2"] < 2.0 * f["dof"]
    assert f["E_end"] == pytest.approx(th * math.exp(width), rel=0.08)


def test_energy_scan_cells():
    """Fig. 4 cells: r0 = 20,000 a0 meets 10 |V(r0)| < E at every energy, and each cell's velocity
    tolerance follows its head-on speed."""
    systems, E, names = I.energy_scan_systems()
    assert len(systems) == 5 * 100 and len(set(names)) == 5
    for s, e in zip(systems, E):
        C4 = 0.5 * s.alpha
        C8 = C4 * C4 / (4 * s.De)
        V = C8 / s.r0 ** 8 - C4 / s.r0 ** 4
        assert 10 * abs(V) < e
        assert s.atol_vel == pytest.approx(1e-10 * math.sqrt(2 * e / s.m_atom), rel=1e-12)
    assert E.min() == pytest.approx(I.kelvin(3e-8)) and E.max() == pytest.approx(I.kelvin(1e-3))


def test_thermal_sweep_cells():
    """Fig. 3 cells: 5 species x 3 temperatures x 2 well depths, r0 = 5000 a0 meeting 10 |V(r0)| < kT,
    velocity tolerance scaled by the cell's thermal speed."""
    systems, cells = I.thermal_sweep_systems()
    assert len(systems) == 30 and len(set(cells)) == 30
    for s, (sp, T, De) in zip(systems, cells):
        assert s.De == pytest.approx(I.kelvin(De))
        C4 = 0.5 * s.alpha
        assert 10 * C4 / s.r0 ** 4 < I.kelvin(T)
        assert s.atol_vel == pytest.approx(1e-10 * math.sqrt(I.kelvin(T) / s.m_atom), rel=1e-12)
