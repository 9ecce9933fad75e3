"""Pins of the CPU oracle to results fixed by the paper and by mathematics (no GPU needed).

Each test checks the oracle against something other than itself: a closed form, an invariant, a
library routine applied to a special case, or a brute-force integration. Together they are chosen so
that a dropped term, a wrong sign or index, or a wrong tableau entry in the oracle fails one of them.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2509_15117_gb300 import inputs as I
from tests import twobody as TB


def rb_system(**kw):
    base = dict(species="Rb", De_K=1.0, q=0.1, a=0.0, r0=5000.0, t_max_s=1e-3, E_K=1.5e-6)
    base.update(kw)
    return I.make_system(**base)


# ---------------------------------------------------------------- P1: potential (text after Eq. 1)

def test_potential_minimum_is_minus_De():
    """C8 = C4^2/(4 D_e) puts the minimum of V = C8/r^8 - C4/r^4 at r_e^4 = C4/(2 D_e) with V = -D_e."""
    for sp in I.SPECIES:
        for De_K in (0.1, 1.0, 100.0):
            d = rb_system(species=sp, De_K=De_K).as_dict()
            C4 = 0.5 * d["alpha"]
            re = (C4 / (2.0 * d["De"])) ** 0.25
            V, dV = O.potential(d, re)
            assert V == pytest.approx(-d["De"], rel=1e-13)
            assert abs(dV) <= 1e-12 * (4.0 * C4 / re ** 5)
            # repulsive inside, attractive outside
            assert O.potential(d, 0.9 * re)[1] < 0.0 < O.potential(d, 1.1 * re)[1]
            # long range tail is -C4/r^4
            Vfar, _ = O.potential(d, 1e4)
            assert Vfar == pytest.approx(-C4 / 1e16, rel=1e-9)


def test_rb_constants_quoted():
    """Rb with alpha = 319 a.u.: C4 = 159.5; D_e = 1 K gives C8 ~ 2.008e9 and r_e ~ 70.8 a0."""
    d = rb_system().as_dict()
    C4 = 0.5 * d["alpha"]
    assert C4 == 159.5
    C8 = C4 ** 2 / (4.0 * d["De"])
    assert C8 == pytest.approx(2.008e9, rel=1e-3)
    re = (C4 / (2.0 * d["De"])) ** 0.25
    assert re == pytest.approx(70.8, rel=2e-3)


# ---------------------------------------------------------------- P2: Dormand-Prince 5(4)

def test_dp5_exponential_and_oscillator_adaptive():
    for lam in (-1.0, 0.7):
        y, ns, nr = O.test_solve(0, lam, 3.0, [1.0], rtol=1e-10, atol=1e-14, hmax=1.0)
        assert y[0] == pytest.approx(math.exp(lam * 3.0), rel=3e-9)
    w = 2.0
    T = 10.0
    y, ns, nr = O.test_solve(1, w, T, [1.0, 0.0], rtol=1e-10, atol=1e-14, hmax=10.0)
    assert y[0] == pytest.approx(math.cos(w * T), abs=5e-9)
    assert y[1] == pytest.approx(-w * math.sin(w * T), abs=1e-8)


def _fixed_error(n):
    p = 1.0
    T = 1.0
    y, err = O.test_fixed(2, p, T / n, n, [1.0, 0.0, 1.0, 0.0, 1.0, 0.0])
    exact = []
    for m in range(3):
        w = p * (m + 1)
        exact += [math.cos(w * T), -w * math.sin(w * T)]
    return np.max(np.abs(y - np.array(exact))), np.max(np.abs(err))


def test_dp5_convergence_orders():
    """Global error of the fifth-order solution falls as h^5; the embedded estimate (the difference
    between the fifth- and fourth-order solutions over one step) falls as h^5 too."""
    e1, l1 = _fixed_error(40)
    e2, l2 = _fixed_error(80)
    e3, l3 = _fixed_error(160)
    assert 28.0 < e2 / e3 < 35.0 and 28.0 < e1 / e2 < 36.0
    assert 28.0 < l1 / l2 < 35.0 and 28.0 < l2 / l3 < 35.0


def test_dp5_step_count_scaling():
    """With per-step error control the number of steps grows like rtol^(-1/5)."""
    _, n1, _ = O.test_solve(1, 1.0, 50.0, [1.0, 0.0], rtol=1e-6, atol=1e-20, hmax=100.0)
    _, n2, _ = O.test_solve(1, 1.0, 50.0, [1.0, 0.0], rtol=1e-11, atol=1e-20, hmax=100.0)
    assert 7.0 < n2 / n1 < 14.0


def test_dense_output_order_and_endpoint():
    """The continuous extension reproduces the step end at s = 1 and is accurate to O(h^5) inside."""
    y0 = [1.0, 0.0, 1.0, 0.0, 1.0, 0.0]
    for s in (0.3, 0.5, 0.77):
        errs = []
        for h in (0.2, 0.1, 0.05):
            out = O.test_dense(2, 1.0, h, s, y0)
            ex = []
            for m in range(3):
                w = m + 1.0
                ex += [math.cos(w * s * h), -w * math.sin(w * s * h)]
            errs.append(np.max(np.abs(out - np.array(ex))))
        assert 22.0 < errs[0] / errs[1] < 40.0 and 22.0 < errs[1] / errs[2] < 40.0
    end = O.test_dense(2, 1.0, 0.1, 1.0, y0)
    ystep, _ = O.test_fixed(2, 1.0, 0.1, 1, y0)
    assert np.max(np.abs(end - ystep)) < 1e-15


# ---------------------------------------------------------------- P3: invariants, trap off

def _total_energy(d, y):
    C4, C8 = TB.coefficients(d["alpha"], d["De"])
    r = np.linalg.norm(y[6:9] - y[0:3])
    return (0.5 * d["m_atom"] * y[9:12] @ y[9:12] + 0.5 * d["m_ion"] * y[3:6] @ y[3:6]
            + TB.V(r, C4, C8))


def _off_axis_ic(r0, v0, b, direction=(0.3, -0.5, 0.81)):
    vhat = np.array(direction) / np.linalg.norm(direction)
    e1 = np.cross(vhat, [0.0, 0.0, 1.0])
    e1 /= np.linalg.norm(e1)
    y = np.zeros(12)
    y[6:9] = b * e1 - math.sqrt(r0 * r0 - b * b) * vhat
    y[9:12] = v0 * vhat
    return y


def test_conservation_trap_off():
    """Trap off (a = q = 0): total energy, momentum and angular momentum are conserved. The error of
    an invariant is set by the tolerance at the bounce, where the relative speed is
    w_max = sqrt(2 (D_e + E) / mu): it must stay below 10 rtol on that scale and shrink with rtol."""
    errs = {}
    for rtol in (1e-10, 1e-12):
        sysd = rb_system(q=0.0, rtol=rtol)
        d = sysd.as_dict()
        E = I.kelvin(1.5e-6)
        v0 = I.speed_for_energy(E, d["m_atom"])
        mu = d["m_ion"] * d["m_atom"] / (d["m_ion"] + d["m_atom"])
        wmax = math.sqrt(2.0 * (d["De"] + E) / mu)
        ys = np.stack([_off_axis_ic(d["r0"], v0, b) for b in (0.0, 150.0, 400.0, 900.0)])
        res = O.run_batch([d], ys, np.zeros(len(ys)))
        worst = 0.0
        for y0, r in zip(ys, res):
            assert r["status"] == O.EXIT
            yf = r["y_final"]
            eE = abs(_total_energy(d, yf) - _total_energy(d, y0)) / (0.5 * mu * wmax ** 2)
            P0 = d["m_atom"] * y0[9:12] + d["m_ion"] * y0[3:6]
            Pf = d["m_atom"] * yf[9:12] + d["m_ion"] * yf[3:6]
            eP = np.max(np.abs(Pf - P0)) / (mu * wmax)
            L0 = d["m_atom"] * np.cross(y0[6:9], y0[9:12]) + d["m_ion"] * np.cross(y0[0:3], y0[3:6])
            Lf = d["m_atom"] * np.cross(yf[6:9], yf[9:12]) + d["m_ion"] * np.cross(yf[0:3], yf[3:6])
            eL = np.max(np.abs(Lf - L0)) / (mu * v0 * d["r0"])
            worst = max(worst, eE, eP, eL)
        assert worst < 10.0 * rtol
        errs[rtol] = worst
    assert errs[1e-12] < errs[1e-10] / 20.0


def _rel(a, b):
    return abs(a / b - 1.0)


@pytest.mark.parametrize("species", ["Li", "Rb", "Cs"])
def test_head_on_trap_off_elastic_limit(species):
    """Head-on with the trap off is a 1D elastic collision, exact at the outward crossing of r0:
    theta_s = pi, dp = 2 mu v0, dE_ion = 4 m_a m_i/(m_a+m_i)^2 E, one bounce, t_f by quadrature.
    theta_s = pi holds to rounding by symmetry; the other observables converge to the exact values in
    proportion to rtol (the bounce raises the relative speed ~10^3-fold over v0, so the asymptotic
    observables carry ~10^5 rtol)."""
    errs = {}
    for rtol in (1e-10, 1e-12):
        sysd = rb_system(species=species, q=0.0, rtol=rtol)
        d = sysd.as_dict()
        E = I.kelvin(1.5e-6)
        v0 = I.speed_for_energy(E, d["m_atom"])
        th, ph = np.array([0.3, 1.1]), np.array([0.2, 1.4])
        y0 = I.head_on(th, ph, d["r0"], v0)
        res = O.run_batch([d], y0, np.zeros(2))
        mi, ma = d["m_ion"], d["m_atom"]
        mu = mi * ma / (mi + ma)
        tf_exact, _, _, _ = TB.relative_passage(d["alpha"], d["De"], mu, d["r0"], v0, 0.0)
        worst = 0.0
        for r in res:
            assert r["status"] == O.EXIT and r["n_bounce"] == 1
            assert abs(r["theta_s"] - math.pi) < 1e-11
            worst = max(worst, _rel(r["dp"], 2.0 * mu * v0),
                        _rel(r["dE_ion"], 4.0 * ma * mi / (ma + mi) ** 2 * E),
                        _rel(r["t_final"], tf_exact))
        assert worst < 2e6 * rtol
        errs[rtol] = worst
    assert errs[1e-12] < errs[1e-10] / 20.0
    if species == "Rb":
        assert 2.0 * mu * v0 == pytest.approx(1.6366e-3, rel=1e-4)


@pytest.mark.parametrize("b", [80.0, 250.0, 600.0, 1500.0])
def test_off_axis_trap_off_deflection(b):
    """Off-axis with the trap off: the crossing state follows from the quadrature of the C8-C4 orbit
    and two-body kinematics (tests/twobody.py); the oracle converges to it in proportion to rtol."""
    errs = {}
    for rtol in (1e-10, 1e-12):
        d = rb_system(q=0.0, rtol=rtol).as_dict()
        v0 = I.speed_for_energy(I.kelvin(1.5e-6), d["m_atom"])
        y0 = _off_axis_ic(d["r0"], v0, b)
        r = O.run_batch([d], y0[None, :], np.zeros(1))[0]
        ex = TB.trap_off_outcome(d["alpha"], d["De"], d["m_ion"], d["m_atom"], y0)
        assert r["status"] == O.EXIT
        worst = max(_rel(r["theta_s"], ex["theta_s"]), _rel(r["dp"], ex["dp"]),
                    _rel(r["dE_ion"], ex["dE_ion"]), _rel(r["t_final"], ex["t_f"]),
                    np.max(np.abs(r["y_final"][9:12] - ex["v_af"])) / v0)
        assert worst < 3e6 * rtol
        errs[rtol] = worst
        mu = d["m_ion"] * d["m_atom"] / (d["m_ion"] + d["m_atom"])
        assert r["dp"] <= 2.0 * mu * v0 * (1 + 1e-12)
    assert errs[1e-12] < errs[1e-10] / 20.0


# ---------------------------------------------------------------- P6: free ion, Mathieu equation

def _hill_beta(a, q, nmax=25):
    """Characteristic exponent beta of x'' + (a + 2 q cos 2 tau) x = 0 by Hill's method: with
    x = sum_n c_n exp(i (beta + 2n) tau), a is an eigenvalue of the symmetric tridiagonal matrix
    diag((beta + 2n)^2) - q (sub + super diagonal). The lowest band rises monotonically on [0, 1]."""
    from scipy import optimize
    ns = np.arange(-nmax, nmax + 1)

    def low(beta):
        Tm = np.diag((beta + 2.0 * ns) ** 2) - q * (np.eye(len(ns), k=1) + np.eye(len(ns), k=-1))
        return np.linalg.eigvalsh(Tm)[0] - a
    return optimize.brentq(low, 0.0, 1.0, xtol=1e-15, rtol=1e-15)


def _free_ion_system(q, a, rf_sign=1):
    sysd = rb_system(q=q, a=a, rf_sign=rf_sign, alpha=0.0)
    sysd.r0 = 1e30  # no exit event
    return sysd


@pytest.mark.parametrize("q,a", [(0.1, 0.0), (0.3, 0.0), (0.2, -0.001), (0.05, 0.002)])
def test_free_ion_monodromy_trace(q, a):
    """Atom absent (alpha = 0): the ion obeys Mathieu's equation in tau = Omega t / 2. Over one rf
    period the monodromy trace is 2 cos(pi beta), beta from Hill's method."""
    sysd = _free_ion_system(q, a)
    d = sysd.as_dict()
    Om = d["Omega"]
    T = 2.0 * math.pi / Om
    d["t_max"] = T
    d["atol_vel"] = 1e-10 * Om
    w = 0.5 * Om
    ys = np.zeros((4, 12))
    ys[:, 6] = 1e6  # distant atom, never interacts
    ys[0, 0] = 1.0          # x axis, position start
    ys[1, 3] = w            # x axis, velocity start (unit in tau)
    ys[2, 1] = 1.0          # y axis
    ys[3, 4] = w
    res = O.run_batch([d], ys, np.zeros(4))
    assert all(r["status"] & O.TMAX for r in res)
    beta = _hill_beta(a, q)
    for ax, (p, v) in enumerate([(0, 1), (2, 3)]):
        trace = res[p]["y_final"][ax] + res[v]["y_final"][3 + ax] / w
        assert trace == pytest.approx(2.0 * math.cos(math.pi * beta), abs=1e-9)
    # small-q secular frequency of the paper: omega = Omega/2 sqrt(a + q^2/2)
    if a == 0.0 and q <= 0.1:
        assert beta == pytest.approx(math.sqrt(a + q * q / 2.0), rel=2e-3)


def test_trap_force_sign_at_phase_zero():
    """Eq. 1 as printed: at phase 0 the ion's restoring constant is (Omega^2/4)(a + 2q)."""
    for sign in (1, -1):
        d = _free_ion_system(0.1, 0.0, rf_sign=sign).as_dict()
        y = np.zeros(12)
        y[0] = 1.0
        y[6] = 1e6
        f = O.rhs(d, 0.0, 0.0, y)
        assert f[3] == pytest.approx(-(d["Omega"] ** 2 / 4.0) * (2.0 * sign * 0.1), rel=1e-14)
        assert f[4] == 0.0 and f[9] == 0.0


def test_static_trap_ion_energy_conserved():
    """q = 0, a > 0: the free ion is a harmonic oscillator with omega^2 = a Omega^2/4 in x and y and
    is unconfined... in z a_z = -2a is repulsive; use x, y only. E_ion = kinetic + trap term is
    conserved and equals m omega^2 X^2 / 2 for a start at rest at X."""
    d = _free_ion_system(0.0, 0.004).as_dict()
    d["t_max"] = 3.0 * 2.0 * math.pi / d["Omega"]
    d["atol_vel"] = 1e-10 * d["Omega"]
    y = np.zeros(12)
    y[0], y[1] = 2.0, -1.5
    y[6] = 1e6
    r = O.run_batch([d], y[None, :], np.zeros(1))[0]
    om2 = 0.004 * d["Omega"] ** 2 / 4.0
    E0 = 0.5 * d["m_ion"] * om2 * (2.0 ** 2 + 1.5 ** 2)
    assert O.ion_energy(d, 0.0, 0.0, y) == pytest.approx(E0, rel=1e-14)
    assert abs(r["dE_ion"]) < 1e-9 * E0
    x = r["y_final"][0]
    assert x == pytest.approx(2.0 * math.cos(math.sqrt(om2) * d["t_max"]), abs=1e-8)


def test_ion_energy_balance_with_rf():
    """Energy balance of the driven ion: dE_ion/dt = dU/dt at fixed x, so E_ion(T) - E_ion(0) equals
    the time integral of -(m Omega^3/4) s q_j sin(Omega t + phi0) x_j^2 along the path (atom absent).
    Checks the trap term of E_ion against the force used in the equations of motion."""
    q, phi0 = 0.2, 0.4
    d = _free_ion_system(q, 0.0).as_dict()
    d["atol_vel"] = 1e-10 * d["Omega"]
    T = 2.0 * math.pi / d["Omega"]
    y = np.zeros(12)
    y[0], y[1] = 1.0, 0.5
    y[3] = 0.1 * d["Omega"]
    y[6] = 1e6
    nseg = 400
    ts = np.linspace(0.0, 1.3 * T, nseg + 1)
    path = [y.copy()]
    cur = y.copy()
    for k in range(nseg):
        cur, _, _ = O.ionatom_segment(d, phi0, ts[k], ts[k + 1], cur)
        path.append(cur.copy())
    path = np.array(path)
    qv = np.array(d["q"])
    integrand = -(d["m_ion"] * d["Omega"] ** 3 / 4.0) * np.sin(d["Omega"] * ts + phi0) * (
        (qv[None, :] * path[:, 0:3] ** 2).sum(axis=1))
    from scipy.integrate import simpson
    work = simpson(integrand, x=ts)
    dE = O.ion_energy(d, phi0, ts[-1], path[-1]) - O.ion_energy(d, phi0, 0.0, path[0])
    scale = np.max(np.abs(integrand)) * ts[-1]
    assert dE == pytest.approx(work, abs=1e-7 * scale)


# ---------------------------------------------------------------- bounce counting on a bound orbit

def test_bounce_count_bound_orbit():
    """Trap off, negative relative energy: the pair oscillates radially with the period of the
    quadrature; a pericentre (bounce) is counted once per period."""
    d = rb_system(q=0.0).as_dict()
    d["r0"] = 1e30
    mi, ma = d["m_ion"], d["m_atom"]
    mu = mi * ma / (mi + ma)
    C4, C8 = TB.coefficients(d["alpha"], d["De"])
    r_start = 400.0
    E_rel = TB.V(r_start, C4, C8) * 0.999  # just below the start potential: nearly at rest
    Tr, rin, rout = TB.radial_period(d["alpha"], d["De"], mu, E_rel)
    # start at r_start moving inward with the speed that gives E_rel (centre of mass at rest)
    w = math.sqrt(2.0 * (E_rel - TB.V(r_start, C4, C8)) / mu)
    y = np.zeros(12)
    y[6] = r_start * ma / (mi + ma) * 0 + r_start
    y[9] = -w * mi / (mi + ma)
    y[3] = +w * ma / (mi + ma)
    k = 6
    # time to first pericentre from r_start
    t_in = TB.relative_passage(d["alpha"], d["De"], mu, r_start, w, 0.0)[0] / 2.0
    d["t_max"] = t_in + (k - 0.5) * Tr
    d["atol_vel"] = 1e-10 * math.sqrt(2 * d["De"] / mu)
    r = O.run_batch([d], y[None, :], np.zeros(1))[0]
    assert r["status"] & O.TMAX
    assert r["n_bounce"] == k
    assert r["status"] & O.COMPLEX
    assert r["t_first_bounce"] == pytest.approx(t_in, rel=1e-3)
    assert r["t_last_bounce"] == pytest.approx(t_in + (k - 1) * Tr, rel=1e-3)


# ---------------------------------------------------------------- P7: brute force, trap on

def _rk4_brute(d, phi0, y0, t1, nsteps):
    """Classical fixed-step RK4 on Eq. 1 (independent restatement), vectorised over trajectories."""
    C4, C8 = TB.coefficients(d["alpha"], d["De"])
    mi, ma, Om = d["m_ion"], d["m_atom"], d["Omega"]
    av, qv = np.array(d["a"]), np.array(d["q"])
    s = float(d["rf_sign"])

    def f(t, Y):
        xi, vi, xa, va = Y[:, 0:3], Y[:, 3:6], Y[:, 6:9], Y[:, 9:12]
        dd = xa - xi
        r2 = np.sum(dd * dd, axis=1, keepdims=True)
        g = 8.0 * C8 / r2 ** 5 - 4.0 * C4 / r2 ** 3  # -V'(r)/r
        c = s * np.cos(Om * t + phi0)[:, None]
        ai = -(g / mi) * dd - (Om * Om / 4.0) * (av[None, :] + 2.0 * qv[None, :] * c) * xi
        aa = (g / ma) * dd
        return np.concatenate([vi, ai, va, aa], axis=1)

    Y = np.array(y0, dtype=np.float64)
    h = t1 / nsteps
    t = 0.0
    for k in range(nsteps):
        k1 = f(t, Y)
        k2 = f(t + 0.5 * h, Y + 0.5 * h * k1)
        k3 = f(t + 0.5 * h, Y + 0.5 * h * k2)
        k4 = f(t + h, Y + h * k3)
        Y = Y + (h / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
        t = (k + 1) * h
    return Y


@pytest.mark.slow
def test_rk4_brute_force_coupled_bounce():
    """Trap on, atom starting at 300 a0 inside the well region: one bounce over a fixed time window.
    Richardson-extrapolated fixed-step RK4 (h and h/2) agrees with the adaptive DP5 oracle."""
    d = rb_system(q=0.1).as_dict()
    mi, ma = d["m_ion"], d["m_atom"]
    n = 6
    rng = np.random.default_rng(7)
    y0 = np.zeros((n, 12))
    phi0 = rng.random(n) * 2 * math.pi
    C4, C8 = TB.coefficients(d["alpha"], d["De"])
    mu = mi * ma / (mi + ma)
    r_s = 300.0
    for k in range(n):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        b = 20.0 * k
        perp = np.cross(u, [0.0, 0.0, 1.0])
        perp /= np.linalg.norm(perp)
        y0[k, 6:9] = r_s * u + b * perp
        w = math.sqrt(2.0 * (I.kelvin(1.5e-6) - TB.V(r_s, C4, C8)) / mu)
        y0[k, 9:12] = -w * u
    t1 = 3.2e8
    Ya = _rk4_brute(d, phi0, y0, t1, 16000)
    Yb = _rk4_brute(d, phi0, y0, t1, 32000)
    Yx = Yb + (Yb - Ya) / 15.0
    wmax = math.sqrt(2.0 * (d["De"] + I.kelvin(1.5e-6)) / mu)
    # the brute force itself is converged far below the tolerance checked
    assert np.max(np.abs(Yb - Ya)[:, 9:12]) / 15.0 < 0.05 * 10.0 * d["rtol"] * wmax
    for k in range(n):
        yo, _, _ = O.ionatom_segment(d, phi0[k], 0.0, t1, y0[k])
        # errors measured on the bounce scale: 10 rtol of the largest relative speed, and of the
        # distance travelled at that speed over the window for positions
        assert np.max(np.abs(yo[9:12] - Yx[k, 9:12])) < 10.0 * d["rtol"] * wmax
        assert np.max(np.abs(yo[3:6] - Yx[k, 3:6])) < 10.0 * d["rtol"] * wmax
        assert np.max(np.abs(yo[6:9] - Yx[k, 6:9])) < 10.0 * d["rtol"] * wmax * t1
        assert np.max(np.abs(yo[0:3] - Yx[k, 0:3])) < 10.0 * d["rtol"] * wmax * t1
        # the window really contains the bounce: the pair separated again after approaching
        assert np.linalg.norm(yo[6:9] - yo[0:3]) > 100.0


# ---------------------------------------------------------------- P8: symmetry of the trap

def test_head_on_mirror_symmetry():
    """y -> -y leaves q = (q, -q, 0) invariant: (theta, phi) and (theta, -phi) give identical
    observables. x <-> y maps q to -q, i.e. rf phase + pi: (theta, phi, 0) equals (theta, pi/2 - phi, pi)
    to integration accuracy."""
    systems, y0, phi0, sid = I.c1_workload(8)
    d = systems[0].as_dict()
    v0 = I.speed_for_energy(I.kelvin(1.5e-6), d["m_atom"])
    th = np.array([0.35, 0.9, 1.3])
    ph = np.array([0.2, 0.5, 1.2])
    ya = I.head_on(th, ph, d["r0"], v0)
    yb = I.head_on(th, -ph, d["r0"], v0)
    yc = I.head_on(th, 0.5 * math.pi - ph, d["r0"], v0)
    ra = O.run_batch([d], ya, np.zeros(3))
    rb = O.run_batch([d], yb, np.zeros(3))
    rc = O.run_batch([d], yc, np.full(3, math.pi))
    for k in range(3):
        for f in ("theta_s", "dp", "dE_ion", "t_final"):
            assert rb[k][f] == ra[k][f]
        assert rb[k]["n_bounce"] == ra[k]["n_bounce"]
        if ra[k]["n_bounce"] == 1 and rc[k]["n_bounce"] == 1:
            for f in ("theta_s", "dp", "t_final"):
                assert rc[k][f] == pytest.approx(ra[k][f], rel=1e-8)


# ---------------------------------------------------------------- status / edge cases

def test_status_edge_cases():
    systems, y0, phi0, sid = I.c1_workload(4)
    d = systems[0].as_dict()
    bad = y0[:4].copy()
    bad[0, 9] = np.nan
    bad[1, 6:9] = 0.0  # atom on the ion
    res = O.run_batch([d], bad, np.zeros(4))
    assert res[0]["status"] == O.BAD_IC and res[1]["status"] == O.BAD_IC
    short = dict(d)
    short["t_max"] = 1e9
    r = O.run_batch([short], y0[2:3], np.zeros(1))[0]
    assert r["status"] & O.TMAX and r["t_final"] == 1e9
    capped = dict(d)
    capped["max_attempts"] = 50
    r = O.run_batch([capped], y0[2:3], np.zeros(1))[0]
    assert r["status"] & O.MAX_STEPS and r["n_steps"] + r["n_rej"] == 50
    # sys_id out of range is rejected per trajectory
    r = O.run_batch([d], y0[:2], np.zeros(2), sys_id=np.array([0, 3], dtype=np.int32))
    assert r[0]["status"] == O.EXIT or r[0]["status"] & O.COMPLEX
    assert r[1]["status"] == O.BAD_IC
