"""The oracle's discrete tangent against finite differences of its frozen-step replay (no GPU).

The replay holds the accepted step sizes fixed, so the tangent is the exact derivative of the replayed
map. FP64 rounding is amplified by a bounce (~1e7 at 1 mK, ~1e8 at 1.5 uK), which limits finite
differences of an FP64 replay to ~1e-5; the reference is therefore the same replay in IEEE quad
precision (rounding ~1e-34), central differences at delta and delta/2 combined by Richardson, with a
spacing of 1e-8 of each direction's scale (rad for theta and phi, E, q): the differences are then
converged to many digits (they agree between spacings of 1e-7 and 1e-9), so what remains is the FP64
tangent's own rounding noise. The bar per entry is max(1e-6 |fd|, 4 spread), spread being the
tangent's largest change under six ulp-level perturbations of the initial state; where that spread is
below 1e-7 |fd| the plain 1e-6 bar applies by itself."""
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


def fd_reference(d, y0, hs, mode, dy0, dq, E, q, delta=1e-8):
    """Quad-precision finite differences along the four directions (theta, phi, E, q)."""
    scale = [1.0, 1.0, E, max(q, 1e-3)]
    out = np.zeros((4, 4))
    for k in range(4):
        out[k] = O.fd_extended(d, y0, 0.0, hs, mode, dy0[k] * scale[k], dq[k] * scale[k], delta) / scale[k]
    return out


def tangent_spread(d, y0, hs, mode, dy0, dq, tan, samples=6):
    """Rounding noise of the FP64 tangent: the largest change under `samples` seeded perturbations of the
    initial state by -2..2 ulps in every component, along the same frozen steps (the bounce amplifies
    rounding in the tangent as in the primal)."""
    rng = np.random.default_rng(7)
    sp = np.zeros_like(tan)
    for _ in range(samples):
        yp = np.asarray(y0, dtype=np.float64) * (1.0 + rng.integers(-2, 3, 12) * 2.0 ** -52)
        tp, _ = O.tangent(d, yp, 0.0, hs, mode, dy0, dq)
        sp = np.maximum(sp, np.abs(tp - tan))
    return sp


K_SPREAD = 4.0


def agree(tan, fd, obs, E, q, spread=None, rel=1e-6, k_spread=K_SPREAD):
    """|tan - fd| <= max(rel |fd|, k_spread * spread) + an absolute floor of 1e-13 of each observable per
    unit of direction (for derivatives that vanish by symmetry)."""
    unit = np.array([1.0, 1.0, E, max(q, 1e-3)])
    floor = 1e-13 * np.abs(np.asarray(obs))[None, :] / unit[:, None]
    bar = rel * np.abs(fd)
    if spread is not None:
        bar = np.maximum(bar, k_spread * spread)
    return np.abs(tan - fd) <= bar + floor


# (species, E in K, q, theta, phi): single-bounce head-on trajectories from 1 mK down to the 1.5 uK of
# the differentiation workload, where a bounce amplifies rounding most
CASES = [("Rb", 1e-3, 0.1, 0.7, 0.3), ("Li", 3e-4, 0.1, 1.1, 0.9), ("Cs", 1e-3, 0.2, 0.4, 1.2),
         ("K", 1e-4, 0.1, 0.5, 0.7), ("Rb", 1.5e-6, 0.1, 0.5, 1.0), ("Rb", 1.5e-6, 0.1, 0.2, 1.3)]


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
    # the reference has converged: a spacing ten times smaller changes it far below the bar
    fd2 = fd_reference(d, y0, hs, mode, dy0, dq, E, q, delta=1e-9)
    np.testing.assert_allclose(fd2, fd, rtol=1e-9, atol=0.0)
    spread = tangent_spread(d, y0, hs, mode, dy0, dq, tan)
    ok = agree(tan, fd, obs, E, q, spread)
    assert ok.all(), (np.argwhere(~ok).tolist(), (tan / fd - 1)[~ok], (np.abs(tan - fd) / spread)[~ok])
    # where the tangent's own rounding noise is small, the plain 1e-6 bar holds
    quiet = spread < 1e-7 * np.abs(fd)
    assert np.all(agree(tan, fd, obs, E, q)[quiet])
    print(species, E_K, "entries within 1e-6 of the reference:", float(np.mean(agree(tan, fd, obs, E, q))))


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
