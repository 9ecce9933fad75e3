"""Closed-form and quadrature results for the ion-atom pair with the trap switched off.

With q = a = 0 the ion and atom form an isolated two-body problem: the centre of mass moves
uniformly and the relative coordinate d = x_a - x_i moves in the central potential
V(r) = C8/r^8 - C4/r^4 (text after Eq. 1 of arXiv 2509.15117) with reduced mass
mu = m_a m_i / (m_a + m_i). A relative orbit that enters the sphere |d| = r0 leaves it again at the
mirror image of its entry point about the apse line (time-reversal symmetry of a central force), so
the state at the outward crossing follows from two one-dimensional quadratures:
    t_f       = 2 int_{r_min}^{r0} dr / rdot(r)
    Delta psi = 2 int_{r_min}^{r0} (L / (mu r^2)) dr / rdot(r)
with rdot(r)^2 = 2 (E - V(r)) / mu - L^2 / (mu r)^2 and r_min the first turning point inside r0.
The quadratures use scipy's adaptive Gauss-Kronrod routine after the substitution
r = r_min + u^2, which removes the inverse-square-root endpoint singularity.

Test helper only: independent of both the oracle and the CUDA library.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate, optimize


def coefficients(alpha: float, De: float):
    C4 = 0.5 * alpha
    C8 = C4 * C4 / (4.0 * De) if C4 != 0.0 else 0.0
    return C4, C8


def V(r, C4, C8):
    return C8 / r ** 8 - C4 / r ** 4


def turning_point(E, L, mu, C4, C8, r0):
    """Largest r < r0 with rdot^2(r) = 0 (first turning point met on the way in)."""
    def f(r):
        return 2.0 * (E - V(r, C4, C8)) / mu - (L / (mu * r)) ** 2
    rs = np.geomspace(r0, 1.0, 20000)
    vals = np.array([f(r) for r in rs])
    assert vals[0] > 0.0
    k = int(np.argmax(vals <= 0.0))
    assert k > 0, "no turning point found"
    return optimize.brentq(f, rs[k], rs[k - 1], xtol=1e-15, rtol=1e-15, maxiter=500)


def relative_passage(alpha, De, mu, r0, v, b):
    """Entry at |d| = r0 with relative speed v and impact parameter b. Returns
    (t_f, delta_psi, rdot0, vt): time inside r0, swept polar angle, radial and tangential speed at r0."""
    C4, C8 = coefficients(alpha, De)
    L = mu * b * v
    E = 0.5 * mu * v * v + V(r0, C4, C8)
    rmin = turning_point(E, L, mu, C4, C8, r0)

    def rdot(r):
        val = 2.0 * (E - V(r, C4, C8)) / mu - (L / (mu * r)) ** 2
        return math.sqrt(max(val, 0.0))

    umax = math.sqrt(r0 - rmin)

    def g_t(u):
        if u == 0.0:
            # limit of 2u / rdot(rmin + u^2) as u -> 0
            eps = 1e-7 * umax
            return 2.0 * eps / rdot(rmin + eps * eps)
        return 2.0 * u / rdot(rmin + u * u)

    def g_psi(u):
        r = rmin + u * u
        return g_t(u) * L / (mu * r * r)

    pts = [umax * f for f in (0.01, 0.05, 0.2, 0.5)]
    t_half, _ = integrate.quad(g_t, 0.0, umax, epsabs=0.0, epsrel=2e-14, limit=1000, points=pts)
    psi_half = 0.0
    if L != 0.0:
        psi_half, _ = integrate.quad(g_psi, 0.0, umax, epsabs=0.0, epsrel=2e-14, limit=1000, points=pts)
    vt = L / (mu * r0)
    rdot0 = rdot(r0)
    return 2.0 * t_half, 2.0 * psi_half, rdot0, vt


def trap_off_outcome(alpha, De, m_i, m_a, y0):
    """Exact outcome at the outward crossing for an ion and atom with the trap off.
    y0 = [x_i, v_i, x_a, v_a]. Returns dict with t_f, theta_s, dp, dE_ion, v_af, v_if."""
    y0 = np.asarray(y0, dtype=np.float64)
    xi, vi, xa, va = y0[0:3], y0[3:6], y0[6:9], y0[9:12]
    M = m_i + m_a
    mu = m_i * m_a / M
    d0 = xa - xi
    w0 = va - vi
    r0 = float(np.linalg.norm(d0))
    v = float(np.linalg.norm(w0))
    Vcm = (m_a * va + m_i * vi) / M
    er = d0 / r0
    cross = np.cross(d0, w0)
    b = float(np.linalg.norm(cross)) / v
    t_f, dpsi, rdot0, vt = relative_passage(*_alpha_de(alpha, De), mu, r0, v, b)
    if b == 0.0:
        w_out = -w0
    else:
        n = cross / np.linalg.norm(cross)
        epsi = np.cross(n, er)
        er_f = math.cos(dpsi) * er + math.sin(dpsi) * epsi
        ep_f = -math.sin(dpsi) * er + math.cos(dpsi) * epsi
        w_out = rdot0 * er_f + vt * ep_f
    v_af = Vcm + (m_i / M) * w_out
    v_if = Vcm - (m_a / M) * w_out
    theta = math.atan2(np.linalg.norm(np.cross(va, v_af)), float(np.dot(va, v_af)))
    return {
        "t_f": t_f, "theta_s": theta, "dp": m_a * float(np.linalg.norm(v_af - va)),
        "dE_ion": 0.5 * m_i * float(np.dot(v_if, v_if)) - 0.5 * m_i * float(np.dot(vi, vi)),
        "v_af": v_af, "v_if": v_if,
    }


def _alpha_de(alpha, De):
    return alpha, De


def radial_period(alpha, De, mu, E, L=0.0):
    """Radial period 2 int dr/rdot between the turning points of a bound orbit (E < 0)."""
    C4, C8 = coefficients(alpha, De)

    def f(r):
        return 2.0 * (E - V(r, C4, C8)) / mu - (L / (mu * r)) ** 2
    # bracket: inner wall below r_e, outer turning point above
    re = (C4 / (2.0 * De)) ** 0.25
    rin = optimize.brentq(f, 0.5 * re, re, xtol=1e-15, rtol=1e-15)
    rout = optimize.brentq(f, re, 1e6, xtol=1e-12, rtol=1e-15)
    mid = 0.5 * (rin + rout)

    def seg(a, bnd, sign):
        # substitution around each turning point
        span = abs(bnd - a)
        um = math.sqrt(span)

        def g(u):
            r = a + sign * u * u
            val = f(r)
            if val <= 0.0:
                eps = 1e-7 * um
                r = a + sign * eps * eps
                return 2.0 * eps / math.sqrt(f(r))
            return 2.0 * u / math.sqrt(val)
        return integrate.quad(g, 0.0, um, epsabs=0.0, epsrel=2e-14, limit=1000)[0]
    half = seg(rin, mid, +1.0) + seg(rout, mid, -1.0)
    return 2.0 * half, rin, rout
