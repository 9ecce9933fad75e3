"""The oracle's discrete tangent against finite differences of its frozen-step replay (no GPU).

The replay holds the accepted step sizes fixed, so the tangent is the exact derivative of the replayed
map. FP64 rounding is amplified by a bounce (~1e7 at the noise floor), which limits finite
differences of an FP64 replay to ~1e-5; the reference is therefore the same replay in extended
precision (long double), central differences at delta and delta/2 combined by Richardson. Spacings are
scaled to each direction: 1e-4 rad for theta and phi, 1e-4 of q for q, 1e-6 of E for E (the exit phase Omega t_f moves fastest with E)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2509_15117_gb300 import inputs as I


def make_case(species, E_K, q, theta, phi):
    sysd = I.make_system(species, De_K=1.0, q=q, r0=5000.0, E_K=E_K)
    d = sysd.as_dict()
    E = I.kelvin(E_K)
    v0 = I.speed_for_energy(E, d["m_atom"])
    y0 = I.head_on(np.array([theta]), np.array([phi]), d["r0"], v0)[0]
    seeds = I.head_on_seeds(np.array([theta]), np.array([phi]), d["r0"], v0, E)[0]
    dy0 = np.concatenate([seeds, np.zeros((1, 12))])
    dq = np.zeros((4, 3))
    dq[3] = I.q_direction()
    return d, y0, E, dy0, dq


def fd_reference(d, y0, hs, mode, dy0, dq, E, q):
    """Extended-precision finite differences along the four directions (theta, phi, E, q)."""
    scale = [1.0, 1.0, E, max(q, 1e-3)]
    delta = [1e-4, 1e-4, 1e-6, 1e-4]
    out = np.zeros((4, 4))
    for k in range(4):
        out[k] = O.fd_extended(d, y0, 0.0, hs, mode, dy0[k] * scale[k], dq[k] * scale[k], delta[k]) / scale[k]
    return out


def tangent_spread(d, y0, hs, mode, dy0, dq, tan):
    """Rounding noise of the FP64 tangent: its change under two ulp-level perturbations of the initial
    state along the same frozen steps (the bounce amplifies rounding in the tangent as in the primal)."""
    sp = np.zeros_like(tan)
    for c, f in ((slice(6, 9), 1.0 + 2.0 ** -51), (slice(9, 12), 1.0 - 2.0 ** -51)):
        yp = np.array(y0, copy=True)
        yp[c] *= f
        tp, _ = O.tangent(d, yp, 0.0, hs, mode, dy0, dq)
        sp = np.maximum(sp, np.abs(tp - tan))
    return sp


def agree(tan, fd, obs, E, q, spread=None, rel=1e-6, k_spread=30.0):
    """|tan - fd| <= max(rel |fd|, k_spread * spread) + an absolute floor of 1e-9 of each observable per
    unit of direction."""
    unit = np.array([1.0, 1.0, E, max(q, 1e-3)])
    floor = 1e-9 * np.abs(np.asarray(obs))[None, :] / unit[:, None]
    bar = rel * np.abs(fd)
    if spread is not None:
        bar = np.maximum(bar, k_spread * spread)
    return np.abs(tan - fd) <= bar + floor


CASES = [("Rb", 1e-3, 0.1, 0.7, 0.3), ("Li", 3e-4, 0.1, 1.1, 0.9), ("Cs", 1e-3, 0.2, 0.4, 1.2),
         ("K", 1e-4, 0.1, 0.5, 0.7)]


@pytest.mark.parametrize("species,E_K,q,theta,phi", CASES)
def test_tangent_matches_extended_precision_finite_differences(species, E_K, q, theta, phi):
    d, y0, E, dy0, dq = make_case(species, E_K, q, theta, phi)
    rec, hs, mode = O.trajectory_steps(d, y0, 0.0)
    assert rec["status"] == O.EXIT and mode == 0 and rec["n_bounce"] == 1
    # the FP64 replay reproduces the adaptive run bit for bit
    obs, yf = O.replay(d, y0, 0.0, hs, mode)
    np.testing.assert_array_equal(yf, rec["y_final"])
    assert obs[3] == rec["t_final"]
    tan, _ = O.tangent(d, y0, 0.0, hs, mode, dy0, dq)
    fd = fd_reference(d, y0, hs, mode, dy0, dq, E, q)
    spread = tangent_spread(d, y0, hs, mode, dy0, dq, tan)
    ok = agree(tan, fd, obs, E, q, spread)
    assert ok.all(), (np.argwhere(~ok).tolist(), (tan / fd - 1)[~ok])
    # most entries meet the plain 1e-6 bar
    assert np.mean(agree(tan, fd, obs, E, q)) >= 0.75


def test_tangent_trap_off_symmetry():
    """Trap off: the head-on observables cannot depend on the direction of approach, so their theta and
    phi derivatives vanish (to rounding), while the energy derivative does not."""
    d, y0, E, dy0, dq = make_case("Rb", 1e-3, 0.0, 0.9, 0.5)
    rec, hs, mode = O.trajectory_steps(d, y0, 0.0)
    tan, _ = O.tangent(d, y0, 0.0, hs, mode, dy0[:3], dq[:3])
    obs = [rec["theta_s"], rec["dp"], abs(rec["dE_ion"]), rec["t_final"]]
    for k in (0, 1):
        assert np.all(np.abs(tan[k]) <= 1e-9 * np.array(obs))
    assert np.all(np.abs(tan[2][1:]) > 1e-3 * np.array(obs[1:]) / E)
