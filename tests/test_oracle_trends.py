"""Qualitative claims of the paper checked on the oracle (CPU only). These are sanity checks of the
method as implemented, not parity: the paper prints no numbers for them.

Fig. 1 discussion, on the Yb+-Rb head-on map at 1.5 uK:
- there is a regular region where the atom leaves after a single bounce;
- the line phi = pi/4 is dominated by complexes. There x = y, so the micromotion that q_x = -q_y
  drives is perpendicular to the incoming velocity.

Near the z axis the trap has no rf component (q_z = 0), so atoms arriving there meet no micromotion
and leave after one bounce.

Fig. 4 inset: with Omega fixed, the complex probability rises with q_x.
Fig. 4 discussion: a fixed initial rf phase makes the complex probability oscillate with energy.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2509_15117_gb300 import inputs as I


@pytest.fixture(scope="module")
def maps():
    systems, y0, phi0, sid = I.c1_workload(32)
    descs = [s.as_dict() for s in systems]
    out = {}
    for k in range(4):  # phases k pi/4; k + 4 is the mirror image phi -> pi/2 - phi
        r = O.run_batch(descs, y0, np.full(len(phi0), k * math.pi / 4), sid)
        out[k] = r["n_bounce"].reshape(32, 32)  # [theta index, phi index]
    return out


def test_phi_quarter_pi_line_is_complex_dominated(maps):
    for k, nb in maps.items():
        cx = nb >= 2
        diag = cx[:, 15:17].mean()  # the two phi columns that bracket pi/4
        assert diag > 0.5 and diag > cx.mean(), (k, diag, cx.mean())


def test_regular_region_and_the_z_axis(maps):
    for k, nb in maps.items():
        assert np.mean(nb == 1) > 0.3, k
        assert np.all(nb[:3] == 1), k  # theta < 0.13 rad: within 7 degrees of the z axis


def test_complex_probability_rises_with_q():
    """Fig. 4 inset: for Yb+-Li at fixed Omega, raising q_x raises the complex probability. Head-on at
    0.3 uK (near Li's threshold), r0 = 20,000 a0, random rf phase, 600 trajectories per q drawn by the
    oracle's sampler."""
    p = []
    for q in (0.05, 0.1, 0.2, 0.3):
        d = I.make_system("Li", q=q, r0=20000.0, E_K=0.3e-6, t_max_s=3e-3).as_dict()
        y, ph = O.sample_ics(O.make_sampler(O.SAMPLE_HEAD_ON, d, 77, E=I.kelvin(0.3e-6)), 0, 600)
        p.append(float(np.mean(O.run_batch([d], y, ph)["n_bounce"] >= 2)))
    assert all(a < b for a, b in zip(p, p[1:])), p
    assert p[0] < 0.1 < 0.2 < p[-1], p


def test_fixed_rf_phase_makes_p_oscillate_with_energy():
    """Fig. 4 discussion: with a fixed initial rf phase the complex probability oscillates by about
    +-0.1 as the energy varies (the phase at impact moves with the approach time r0/v0); a random
    phase averages the oscillation out. Yb+-Li, q = 0.1, r0 = 20,000 a0, 12 energies over
    0.25-0.35 uK, 300 trajectories each; the residual about a linear trend is compared with the
    binomial noise."""
    Es = np.linspace(0.25, 0.35, 12)
    resid_std = {}
    for rand in (False, True):
        P = []
        for E_uK in Es:
            d = I.make_system("Li", q=0.1, r0=20000.0, E_K=E_uK * 1e-6, t_max_s=3e-3).as_dict()
            smp = O.make_sampler(O.SAMPLE_HEAD_ON, d, 78, E=I.kelvin(E_uK * 1e-6), random_phase=rand, phase=0.0)
            y, ph = O.sample_ics(smp, 0, 300)
            P.append(float(np.mean(O.run_batch([d], y, ph)["n_bounce"] >= 2)))
        P = np.array(P)
        resid = P - np.polyval(np.polyfit(Es, P, 1), Es)
        binom = math.sqrt(float(np.mean(P * (1 - P))) / 300)
        resid_std[rand] = (float(resid.std()), binom, float(np.ptp(resid)))
    fixed, rnd = resid_std[False], resid_std[True]
    assert fixed[0] > 3 * fixed[1] and fixed[2] > 0.15, resid_std
    assert rnd[0] < 1.5 * rnd[1], resid_std
