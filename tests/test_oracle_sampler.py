"""Pins of the oracle's counter-based initial-condition samplers (CPU only).

- The generator is pinned to numpy's own Philox4x64-10 bit generator. numpy implements the same
  published definition (Salmon et al., SC'11) and advances its counter before it draws a block.
- Each sampler is pinned to the distributions the paper states, by Kolmogorov-Smirnov tests against
  scipy's distributions and by exact geometric identities:
  - head-on runs: the ion at rest; the atom on the r0 octant moving radially inward at v0;
  - thermal runs: the atom uniform on the r0 sphere with Gaussian velocity components flipped
    inward; the ion Gaussian in an isotropic trap of frequency |q_x| Omega / 2^(3/2);
  - the disk variant: the impact parameter uniform over the disk; the ion with its lowest-order
    micromotion.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2509_15117_gb300 import inputs as I

stats = pytest.importorskip("scipy.stats")

N = 200_000
P_MIN = 1e-4


def rb_desc(r0=5000.0):
    return I.make_system("Rb", r0=r0).as_dict()


def ks_ok(x, dist, *args):
    return stats.kstest(x, dist, args=args).pvalue > P_MIN


# ---------------------------------------------------------------- the generator

@pytest.mark.parametrize("key", [(0, 0), (123, 456), (2 ** 64 - 1, 2 ** 64 - 1), (0x0123456789ABCDEF, 7)])
@pytest.mark.parametrize("ctr", [(0, 0, 0, 0), (41, 3, 5, 7), (2 ** 64 - 1, 9, 0, 2 ** 63)])
def test_philox_block_matches_numpy(key, ctr):
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(ctr, dtype=np.uint64))
    raw = bg.random_raw(8)
    c = list(ctr)
    for blk in range(2):
        # numpy adds one to the 256-bit counter (with carry) before each block
        for w in range(4):
            c[w] = (c[w] + 1) % 2 ** 64
            if c[w] != 0:
                break
        got = O.philox4x64(c, key)
        assert np.array_equal(got, raw[4 * blk:4 * blk + 4]), (key, ctr, blk)


def test_philox_stream_layout():
    out = O.philox4x64_stream(11, 22, 5, 2 ** 40 - 3, 7)
    for j in range(7):
        assert np.array_equal(out[j], O.philox4x64([2 ** 40 - 3 + j, 5, 0, 0], [11, 22]))


def test_uniform_map_and_phase_slot():
    """phi0 = 2 pi u[0], with u = ((x >> 11) | 1) 2^-53 of word 0 of block 0 under key (seed, kind)."""
    d = rb_desc()
    s = O.make_sampler(O.SAMPLE_HEAD_ON, d, seed=99, E=I.kelvin(1.5e-6))
    _, ph = O.sample_ics(s, 1000, 16)
    for i in range(16):
        x = int(O.philox4x64([1000 + i, 0, 0, 0], [99, O.SAMPLE_HEAD_ON])[0])
        u = ((x >> 11) | 1) * 2.0 ** -53
        assert 0.0 < u < 1.0
        assert ph[i] == 2.0 * math.pi * u


def test_chunks_are_slices_of_one_stream():
    d = rb_desc()
    s = O.make_sampler(O.SAMPLE_DISK, d, seed=5, kT=I.kelvin(1e-4), kT_ion=I.kelvin(1e-5), b_max=2000.0,
                       micromotion=True)
    y, ph = O.sample_ics(s, 0, 3000)
    y2, ph2 = O.sample_ics(s, 1234, 1000)
    assert np.array_equal(y[1234:2234], y2) and np.array_equal(ph[1234:2234], ph2)
    s2 = O.make_sampler(O.SAMPLE_DISK, d, seed=6, kT=I.kelvin(1e-4), kT_ion=I.kelvin(1e-5), b_max=2000.0)
    y3, _ = O.sample_ics(s2, 0, 3000)
    assert not np.any(y3[:, 9] == y[:, 9])


# ---------------------------------------------------------------- head-on runs

def test_head_on_octant():
    d = rb_desc()
    E = I.kelvin(1.5e-6)
    s = O.make_sampler(O.SAMPLE_HEAD_ON, d, seed=1, E=E)
    y, ph = O.sample_ics(s, 0, N)
    r0 = d["r0"]
    v0 = math.sqrt(2.0 * E / d["m_atom"])
    assert np.all(y[:, :6] == 0.0)
    xa, va = y[:, 6:9], y[:, 9:12]
    assert np.allclose(np.linalg.norm(xa, axis=1), r0, rtol=1e-14, atol=0)
    assert np.allclose(va, -v0 * xa / r0, rtol=0, atol=1e-14 * v0)
    assert np.all(xa >= 0.0)
    assert ks_ok(xa[:, 2] / r0, "uniform", 0.0, 1.0)          # cos(theta) ~ U(0, 1)
    assert ks_ok(np.arctan2(xa[:, 1], xa[:, 0]), "uniform", 0.0, 0.5 * math.pi)
    assert ks_ok(ph, "uniform", 0.0, 2.0 * math.pi)
    s_fixed = O.make_sampler(O.SAMPLE_HEAD_ON, d, seed=1, E=E, random_phase=False, phase=0.25)
    y_fixed, ph_fixed = O.sample_ics(s_fixed, 0, 100)
    assert np.all(ph_fixed == 0.25) and np.array_equal(y_fixed, y[:100])


# ---------------------------------------------------------------- thermal runs on the sphere

def test_thermal_sphere():
    d = rb_desc()
    kT = I.kelvin(1e-4)
    kTi = I.kelvin(1e-5)
    s = O.make_sampler(O.SAMPLE_SPHERE, d, seed=2, kT=kT, kT_ion=kTi)
    y, ph = O.sample_ics(s, 0, N)
    r0 = d["r0"]
    xa, va = y[:, 6:9], y[:, 9:12]
    xh = xa / r0
    assert np.allclose(np.linalg.norm(xa, axis=1), r0, rtol=1e-14, atol=0)
    assert ks_ok(xh[:, 2], "uniform", -1.0, 2.0)
    assert ks_ok(np.arctan2(xh[:, 1], xh[:, 0]), "uniform", -math.pi, 2.0 * math.pi)
    sig = math.sqrt(kT / d["m_atom"])
    vr = np.sum(va * xh, axis=1)
    assert np.all(vr < 0.0)                                    # negated where it pointed outward
    assert ks_ok(-vr / sig, "halfnorm")                        # |N(0, 1)| along the fixed direction
    assert ks_ok(np.sum(va * va, axis=1) / sig ** 2, "chi2", 3)
    w = abs(d["q"][0]) * d["Omega"] / 2.0 ** 1.5
    sv = math.sqrt(kTi / d["m_ion"])
    for j in range(3):
        assert ks_ok(y[:, j] / (sv / w), "norm")
        assert ks_ok(y[:, 3 + j] / sv, "norm")
    assert ks_ok(ph, "uniform", 0.0, 2.0 * math.pi)
    # the Box-Muller partners of one pair are uncorrelated
    assert abs(np.corrcoef(y[:, 0], y[:, 1])[0, 1]) < 5.0 / math.sqrt(N)


def test_thermal_ion_at_rest_when_cold():
    d = rb_desc()
    s = O.make_sampler(O.SAMPLE_SPHERE, d, seed=3, kT=I.kelvin(1e-4), kT_ion=0.0, micromotion=True)
    y, _ = O.sample_ics(s, 0, 1000)
    assert np.all(y[:, :6] == 0.0)


# ---------------------------------------------------------------- the disk variant

def test_thermal_disk_geometry_and_distributions():
    d = rb_desc()
    kT = I.kelvin(1e-3)
    bmax = 2000.0
    s = O.make_sampler(O.SAMPLE_DISK, d, seed=4, kT=kT, kT_ion=I.kelvin(1e-5), b_max=bmax, micromotion=True)
    y, _ = O.sample_ics(s, 0, N)
    r0 = d["r0"]
    xa, va = y[:, 6:9], y[:, 9:12]
    vh = va / np.linalg.norm(va, axis=1, keepdims=True)
    along = np.sum(xa * vh, axis=1)
    bvec = xa - along[:, None] * vh
    b = np.linalg.norm(bvec, axis=1)
    assert np.allclose(np.linalg.norm(xa, axis=1), r0, rtol=1e-13, atol=0)
    assert np.all(b <= bmax * (1 + 1e-12))
    assert np.allclose(along, -np.sqrt(r0 ** 2 - b ** 2), rtol=0, atol=1e-9 * r0)
    assert ks_ok((b / bmax) ** 2, "uniform", 0.0, 1.0)          # uniform over the disk's area
    sig = math.sqrt(kT / d["m_atom"])
    for j in range(3):
        assert ks_ok(va[:, j] / sig, "norm")
    # azimuth of b about v_hat, measured from e1 = unit(v_hat x z_hat) where |v_hat_z| < 0.9
    m = np.abs(vh[:, 2]) < 0.9
    e1 = np.cross(vh[m], np.array([0.0, 0.0, 1.0]))
    e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
    e2 = np.cross(vh[m], e1)
    psi = np.arctan2(np.sum(bvec[m] * e2, axis=1), np.sum(bvec[m] * e1, axis=1))
    assert ks_ok(psi, "uniform", -math.pi, 2.0 * math.pi)


@pytest.mark.parametrize("phase", [0.0, 0.5 * math.pi])
def test_disk_ion_micromotion(phase):
    """At a fixed rf phase: x_j = X_j (1 + s q_j/2 cos phi0), v_j = V_j (1 + s q_j/2 cos phi0) -
    X_j s (q_j Omega/2) sin phi0, with X, V the secular Gaussians."""
    d = rb_desc()
    kTi = I.kelvin(1e-5)
    s = O.make_sampler(O.SAMPLE_DISK, d, seed=8, kT=I.kelvin(1e-4), kT_ion=kTi, b_max=2000.0,
                       random_phase=False, phase=phase, micromotion=True)
    y, _ = O.sample_ics(s, 0, N)
    w = abs(d["q"][0]) * d["Omega"] / 2.0 ** 1.5
    sv = math.sqrt(kTi / d["m_ion"])
    sx = sv / w
    sg = d["rf_sign"]
    for j in range(3):
        qj = d["q"][j]
        f = 1.0 + sg * 0.5 * qj * math.cos(phase)
        k = sg * 0.5 * qj * d["Omega"] * math.sin(phase)
        assert ks_ok(y[:, j] / (sx * f), "norm")
        sdv = math.sqrt((sv * f) ** 2 + (sx * k) ** 2)
        assert ks_ok(y[:, 3 + j] / sdv, "norm")
        cov = np.mean(y[:, j] * y[:, 3 + j])
        expect = -k * f * sx * sx
        tol = 5.0 * sx * sdv / math.sqrt(N)
        assert abs(cov - expect) < tol, (j, cov, expect, tol)


# ---------------------------------------------------------------- bad parameters

@pytest.mark.parametrize("kw", [
    dict(kind=O.SAMPLE_HEAD_ON, E=0.0),
    dict(kind=O.SAMPLE_SPHERE, kT=0.0),
    dict(kind=O.SAMPLE_SPHERE, kT=1e-9, kT_ion=-1.0),
    dict(kind=O.SAMPLE_DISK, kT=1e-9, b_max=5000.0),
    dict(kind=3, kT=1e-9),
])
def test_bad_parameters(kw):
    d = rb_desc()
    kind = kw.pop("kind")
    with pytest.raises(ValueError):
        O.sample_ics(O.make_sampler(kind, d, seed=1, **kw), 0, 10)


def test_thermal_ion_needs_a_trap():
    d = dict(rb_desc())
    d["q"] = (0.0, 0.0, 0.0)
    with pytest.raises(ValueError):
        O.sample_ics(O.make_sampler(O.SAMPLE_SPHERE, d, seed=1, kT=1e-9, kT_ion=1e-11), 0, 10)
