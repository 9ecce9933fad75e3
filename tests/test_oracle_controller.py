"""Pins of the oracle's step-size controller (CPU; no GPU).

The text after Eq. 1 names the integrator: the adaptive Dormand-Prince 5(4) pair as MATLAB's ode45
runs it (Dormand & Prince 1980; Shampine & Reichelt 1997). The CUDA path takes the same accept/reject
decisions and step sizes as the oracle, so a misread rule of ode45 shared by both would pass every
parity test; these pins tie the oracle's rules to the mathematics instead.

On y' = lam y one attempted step of size h maps y to R(z) y and estimates its error as E(z) y, with
z = lam h and R, E polynomials fixed by the Dormand-Prince tableau. The tests take that step from
SciPy's own Dormand-Prince implementation (``scipy.integrate._ivp.rk.rk_step`` with the RK45
tableau), a library routine independent of the oracle, form ode45's error measure
err = |E y| / max(rtol max(|y|, |R y|), atol), and predict every step size of the oracle's trace from
ode45's rules:
  - accepted step with no failure: h <- h / (1.25 err^(1/5)), but 5 h when that factor exceeds 5;
  - first failure of a step: h <- h max(0.1, 0.8 err^(-1/5));
  - later failures of the same step: h <- h / 2;
  - the step after one that failed starts with the size that was accepted (no growth).
Each constant is then planted wrong in a copy of the oracle (built on the CPU with one macro changed)
and at least one pin must fail.
"""
import math
import tempfile

import numpy as np
import pytest
from scipy.integrate._ivp import rk
from scipy.optimize import brentq

from oracle import oracle as O

LAM = -1.0
RTOL = 1e-8
ATOL = 1e-300   # the error measure is then relative: err = |E(z)| / (rtol max(1, |R(z)|))
HMAX = 1e9      # no step-size cap in play
REL = 1e-12     # step sizes predicted from the recorded error measure, to rounding
REL_ERR = 1e-6  # the error estimate is a difference of O(h) terms: the two implementations' summation
                # orders give it to about 1e-7 relative


def library_step(h: float, y: float = 1.0):
    """One Dormand-Prince step of y' = LAM y by SciPy: (y_new, error estimate)."""
    T = rk.RK45
    K = np.empty((T.n_stages + 1, 1))
    f0 = np.array([LAM * y])
    y_new, _ = rk.rk_step(lambda t, v: LAM * v, 0.0, np.array([y]), f0, h, T.A, T.B, T.C, K)
    err = (K.T @ T.E) * h
    return float(y_new[0]), float(err[0])


def measure(h: float, y: float = 1.0) -> float:
    """ode45's error measure of one step of size h from y."""
    y_new, err = library_step(h, y)
    return abs(err) / max(RTOL * max(abs(y), abs(y_new)), ATOL)


def h_star() -> float:
    """Fixed point of the accepted-step rule: 1.25 err(h)^(1/5) = 1."""
    return brentq(lambda h: measure(h) - 1.25 ** -5, 1e-4, 1.0, xtol=1e-15, rtol=1e-15)


def trace(h0: float, t_end: float, L=None):
    return O.test_trace(0, LAM, t_end, [1.0], rtol=RTOL, atol=ATOL, hmax=HMAX, h0=h0, L=L)


def check_error_measure(L=None):
    """The oracle's recorded error measure of every attempt equals the library step's (ode45's measure
    of SciPy's Dormand-Prince step), from ode45's own first step onwards."""
    tr = trace(0.0, 20.0, L)
    assert len(tr["h"]) > 20
    for t, h, e in zip(tr["t"], tr["h"], tr["err"]):
        y_t = math.exp(LAM * t)  # only the scale of y matters on a linear problem
        assert e == pytest.approx(measure(h, y_t), rel=REL_ERR), (t, h, e)


def check_accepted_rule(L=None):
    """From a tiny first step: every step after an accepted one follows h / (1.25 err^(1/5)) or the
    5x cap, and the accepted sizes settle at the rule's fixed point h*."""
    hs = h_star()
    tr = trace(1e-4 * hs, 40.0, L)
    h, e, acc = tr["h"], tr["err"], tr["acc"]
    assert acc[:-1].all(), "a step was rejected on the way up"
    grow = 0
    for k in range(len(h) - 2):  # the last step is clamped to t_end
        temp = 1.25 * e[k] ** 0.2
        pred = h[k] / temp if temp > 0.2 else 5.0 * h[k]
        grow += temp <= 0.2
        assert h[k + 1] == pytest.approx(pred, rel=REL), (k, h[k], h[k + 1], pred)
    assert grow >= 5, "the 5x cap was never exercised"
    tail = h[len(h) // 2:-1]
    assert np.all(np.abs(tail / hs - 1.0) < REL_ERR), (tail[:3], hs)


def check_first_failure(L=None):
    """An oversized first step fails once and shrinks by max(0.1, 0.8 err^(-1/5)); the next step keeps
    the accepted size."""
    hs = h_star()
    for mult in (3.0, 1.6):
        tr = trace(mult * hs, 10.0, L)
        h, acc = tr["h"], tr["acc"]
        assert not acc[0] and acc[1], (mult, acc[:3])
        e0 = tr["err"][0]
        assert e0 == pytest.approx(measure(h[0]), rel=REL_ERR)
        pred = h[0] * max(0.1, 0.8 * e0 ** -0.2)
        assert h[1] == pytest.approx(pred, rel=REL), (mult, h[:2], pred)
        assert h[2] == h[1], "the step after a failed one grew"


def check_retry_halving(L=None):
    """A hugely oversized first step: the first failure shrinks by the 0.1 floor, every later failure of
    the same step halves, and the accepted size is kept for the next step."""
    hs = h_star()
    tr = trace(3000.0 * hs, 10.0, L)
    h, acc = tr["h"], tr["acc"]
    k_acc = int(np.argmax(acc))
    assert k_acc >= 4, "expected several failures"
    assert 0.8 * tr["err"][0] ** -0.2 < 0.1
    assert h[1] == pytest.approx(0.1 * h[0], rel=REL), h[:2]
    for k in range(1, k_acc):
        assert h[k + 1] == pytest.approx(0.5 * h[k], rel=REL), (k, h[k], h[k + 1])
    assert h[k_acc + 1] == h[k_acc], "the step after a failed one grew"


CHECKS = (check_error_measure, check_accepted_rule, check_first_failure, check_retry_halving)


@pytest.mark.parametrize("check", CHECKS, ids=lambda c: c.__name__)
def test_controller_pins(check):
    check()


@pytest.mark.parametrize("macro,value", [("ORC_CTRL_SAFETY", 0.9), ("ORC_CTRL_GROW_MAX", 10.0),
                                         ("ORC_CTRL_SHRINK_MIN", 0.2), ("ORC_CTRL_RETRY", 0.25),
                                         ("ORC_CTRL_EXPONENT", 0.25), ("ORC_CTRL_SHRINK_SAFETY", 0.9)])
def test_planted_controller_mistakes_fail_a_pin(macro, value):
    with tempfile.TemporaryDirectory() as d:
        L = O.build_variant({macro: value}, d)
        failed = []
        for check in CHECKS:
            try:
                check(L)
            except AssertionError:
                failed.append(check.__name__)
        assert failed, f"{macro} = {value} passes every controller pin"
