"""The oracle's gradient (the transposed Jacobian of the frozen-step map, assembled from its discrete
tangent) against the tangent itself and against symmetries of the equations of motion (no GPU).

With the trap off (a = q = 0) the equations are invariant under a common translation of both particles
and under a common rotation of all positions and velocities; the frozen-step DP5 map and the exit test
|x_a - x_i| = r0 inherit both, and every observable (scattering angle, momentum transfer, ion kinetic
energy change, exit time) is invariant. So the gradient is orthogonal to the generators of these
motions, up to rounding: a dropped term, a wrong sign or a swapped index in the Jacobian breaks that.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2509_15117_gb300 import inputs as I
from tests import test_oracle_tangent as OT


def scales(d, E, q):
    """Characteristic size of each of the 15 inputs: positions r0, velocities v0, q components."""
    v0 = I.speed_for_energy(E, d["m_atom"])
    s = np.array([d["r0"]] * 3 + [v0] * 3 + [d["r0"]] * 3 + [v0] * 3 + [max(q, 1e-3)] * 3)
    return s


def generators(y0):
    """Infinitesimal common translations (3) and rotations (3) of a state, as 12-vectors."""
    g = []
    for k in range(3):
        t = np.zeros(12)
        t[k] = 1.0
        t[6 + k] = 1.0
        g.append(t)
    for k in range(3):
        e = np.zeros(3)
        e[k] = 1.0
        r = np.zeros(12)
        for b in (0, 3, 6, 9):
            r[b:b + 3] = np.cross(e, y0[b:b + 3])
        g.append(r)
    return np.array(g)


def test_gradient_is_the_transposed_tangent():
    d, y0, E, dy0, dq = OT.make_case("Rb", 1e-3, 0.1, 0.7, 0.3)
    rec, hs, mode = O.trajectory_steps(d, y0, 0.0)
    gy, gq = O.gradient(d, y0, 0.0, hs, mode)
    rng = np.random.default_rng(11)
    s = scales(d, E, 0.1)
    v = rng.standard_normal((4, 15)) * s
    tan, _ = O.tangent(d, y0, 0.0, hs, mode, v[:, :12], v[:, 12:])
    G = np.concatenate([gy, gq], axis=1)  # (4 objectives, 15)
    # the two sides sum the same linear map in different orders; a bounce amplifies FP64 rounding
    # by ~1e7, so they agree to ~1e-9 of the sum of magnitudes, while a misplaced entry is O(1) off
    for k in range(4):
        dot = G @ v[k]
        scale = np.abs(G) @ np.abs(v[k])
        np.testing.assert_array_less(np.abs(dot - tan[k]), 1e-7 * scale + 1e-300)


@pytest.mark.parametrize("theta,phi", [(0.9, 0.5), (0.3, 1.2)])
def test_gradient_trap_off_is_orthogonal_to_translations_and_rotations(theta, phi):
    d, y0, E, dy0, dq = OT.make_case("Rb", 1e-3, 0.0, theta, phi)
    # move the ion off the origin so that rotations and translations act on both particles
    y0 = np.array(y0, copy=True)
    y0[0:3] = [37.0, -21.0, 12.5]
    y0[6:9] += y0[0:3]
    rec, hs, mode = O.trajectory_steps(d, y0, 0.0)
    assert rec["status"] == O.EXIT
    gy, _ = O.gradient(d, y0, 0.0, hs, mode)
    s = scales(d, E, 0.0)[:12]
    for gen in generators(y0):
        for m in range(4):
            dot = gy[m] @ gen
            scale = np.linalg.norm(gy[m] * s) * np.linalg.norm(gen / s)
            assert abs(dot) <= 1e-7 * scale, (m, dot, scale)
    # the invariances do not make the gradient vanish
    for m in range(4):
        assert np.linalg.norm(gy[m] * s) > 0.0
