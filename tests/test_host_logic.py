"""Host-side logic that both sides rely on (CPU only): the workload builders, the differentiation
seeds and the queue order."""
import math

import numpy as np
import pytest

from paper_2509_15117_gb300 import inputs as I
from paper_2509_15117_gb300 import schedule as Sch


def test_splitmix64_published_sequence():
    """splitmix64 (Steele, Lea & Flood 2014) seeded with 0 outputs e220a8397b1dcdaf, 6e789e6aa1b965f4,
    06c45d188009454f: the finaliser applied to 1, 2, 3 times the golden-ratio increment."""
    gamma = 0x9E3779B97F4A7C15
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    for k, w in enumerate(want):
        assert I.splitmix64((k * gamma) % 2 ** 64) == w


def test_mixed_sweep_cells():
    cells = I.c4_cells()
    assert len(cells) == 250
    sizes = {c["n"] for c in cells}
    assert sizes <= {4096 * 2 ** k for k in range(7)} and len(sizes) > 3
    assert len({(c["De_K"], c["q"], c["a"], c["species"]) for c in cells}) == 250


def test_octant_grid_is_cell_centred():
    th, ph = I.octant_grid(4)
    step = 0.5 * math.pi / 4
    assert np.allclose(np.unique(th), (np.arange(4) + 0.5) * step)
    assert np.allclose(ph[:4], (np.arange(4) + 0.5) * step)  # phi fastest


def test_head_on_seeds_are_the_derivatives_of_the_initial_state():
    """d y0 / d(theta, phi, E) against central differences of head_on: the seeds feed both the tangent
    kernel and the oracle's tangent, so parity between them cannot catch a wrong seed."""
    d = I.make_system("Rb").as_dict()
    E = I.kelvin(1.5e-6)
    th, ph = np.array([0.3, 1.2]), np.array([0.7, 0.1])
    m = d["m_atom"]
    seeds = I.head_on_seeds(th, ph, d["r0"], math.sqrt(2 * E / m), E)

    def state(t, p, e):
        return I.head_on(t, p, d["r0"], math.sqrt(2 * e / m))

    for k, (dt, dp, de) in enumerate([(1e-6, 0, 0), (0, 1e-6, 0), (0, 0, 1e-6 * E)]):
        fd = (state(th + dt, ph + dp, E + de) - state(th - dt, ph - dp, E - de)) / (2 * (dt + dp + de))
        scale = np.abs(seeds[:, k]).max(axis=1, keepdims=True)
        assert np.all(np.abs(fd - seeds[:, k]) <= 1e-8 * scale), k
    assert np.array_equal(I.q_direction(), [1.0, -1.0, 0.0])


def test_queue_order_puts_costly_systems_first_and_keeps_the_rest_stable():
    systems = [I.make_system(sp, E_K=1e-6) for sp in ("Li", "Cs", "Rb")]
    speeds = [s.atol_vel / 1e-10 for s in systems]
    cost = Sch.system_cost(systems, speeds)
    assert cost[1] > cost[2] > cost[0]  # heavy and slow first
    sid = np.array([0, 1, 2, 1, 0, 2, 1], dtype=np.int32)
    order = Sch.order_by_cost(sid, cost)
    assert sorted(order) == list(range(7))
    assert list(order) == [1, 3, 6, 2, 5, 0, 4]


def test_threshold_order_puts_the_systems_furthest_below_w0_first():
    from paper_2509_15117_gb300 import statistics as St
    c2 = I.c2_systems()
    systems = [s for (_, _, s) in c2]
    energies = [I.kelvin(E) for (_, E, _) in c2]
    w0 = [St.w0_3d(s.m_atom, s.m_ion, s.Omega, s.a[0], s.q[0], 0.5 * s.alpha) for s in systems]
    cost = Sch.system_cost_threshold(energies, w0)
    assert np.allclose(cost, np.asarray(w0) / np.asarray(energies), rtol=0, atol=0)
    names = [(sp, E) for (sp, E, _) in c2]
    ranked = [names[i] for i in np.argsort(-cost, kind="stable")]
    assert ranked[0] == ("Cs", 1e-6) and ranked[-1] == ("Li", 1e-3)
    # at one energy the heavier atom (larger W0^3D) comes first
    at_1uK = [sp for (sp, E) in ranked if E == 1e-6]
    assert at_1uK == ["Cs", "Rb", "K", "Na", "Li"]


def test_part_bounds_cover_the_queue_once():
    import bench
    for n, parts in ((41943040, 20), (1000, 7), (5, 20), (1, 1)):
        b = bench.part_bounds(n, parts)
        assert b[0] == 0 and b[-1] == n and len(b) == parts + 1
        assert np.all(np.diff(b) >= 0)
        assert np.diff(b).max() - np.diff(b).min() <= 1
    b = bench.part_bounds(1000, 5, 0.25)
    assert b[0] == 0 and b[-1] == 1000 and len(b) == 6
    head = np.diff(b)[:-1]
    assert b[-1] - b[-2] == 250 and head.sum() == 750 and head.max() - head.min() <= 1


stats = pytest.importorskip("scipy.stats")


def ks_ok(x, dist, *args):
    return stats.kstest(x, dist, args=args).pvalue > 1e-4


def test_host_thermal_samplers_follow_the_paper():
    """The numpy samplers that feed both sides: atom on the r0 sphere with Gaussian velocity flipped
    inward (thermal-runs paragraph), the disk variant, the ion Gaussian in the secular trap."""
    vth = math.sqrt(I.kelvin(1e-4) / (I.SPECIES["Rb"]["mass_amu"] * I.AMU_TO_ME))
    sysd = I.make_system("Rb", v_scale=vth)
    n = 100_000
    sig = math.sqrt(I.kelvin(1e-4) / sysd.m_atom)
    y, ph = I.thermal_sphere(n, 1, sysd, 1e-4)
    xh = y[:, 6:9] / sysd.r0
    assert np.allclose(np.linalg.norm(xh, axis=1), 1.0, atol=1e-14)
    assert ks_ok(xh[:, 2], "uniform", -1.0, 2.0)
    vr = np.sum(y[:, 9:12] * xh, axis=1)
    assert np.all(vr <= 0.0) and ks_ok(-vr / sig, "halfnorm")
    assert ks_ok(np.sum(y[:, 9:12] ** 2, axis=1) / sig ** 2, "chi2", 3)
    w = I.secular_omega(0.1, sysd.Omega)
    sv = math.sqrt(I.kelvin(10e-6) / sysd.m_ion)
    assert ks_ok(y[:, 0] / (sv / w), "norm") and ks_ok(y[:, 4] / sv, "norm")
    assert ks_ok(ph, "uniform", 0.0, 2 * math.pi)
    yd, _ = I.thermal_disk(n, 2, sysd, 1e-4)
    vh = yd[:, 9:12] / np.linalg.norm(yd[:, 9:12], axis=1, keepdims=True)
    along = np.sum(yd[:, 6:9] * vh, axis=1)
    b = np.linalg.norm(yd[:, 6:9] - along[:, None] * vh, axis=1)
    assert np.allclose(np.linalg.norm(yd[:, 6:9], axis=1), sysd.r0, rtol=1e-12)
    assert ks_ok((b / 2000.0) ** 2, "uniform", 0.0, 1.0)
    cth, phi = I.octant_random(n, 3)
    assert ks_ok(np.cos(cth), "uniform", 0.0, 1.0) and ks_ok(phi, "uniform", 0.0, 0.5 * math.pi)


def test_host_micromotion_covariance():
    """thermal_ion at a fixed phase: cov(x_j, v_j) = -s (q_j Omega / 2) sin(phi0) (1 + s q_j/2 cos phi0)
    sigma_X^2, the lowest-order Mathieu solution."""
    sysd = I.make_system("Rb")
    n = 200_000
    ph = np.full(n, 0.5 * math.pi)
    y = I.thermal_ion(n, np.random.default_rng(4), sysd.m_ion, 1e-5, sysd.q, sysd.Omega, ph)
    sx = math.sqrt(I.kelvin(1e-5) / (sysd.m_ion * I.secular_omega(0.1, sysd.Omega) ** 2))
    sv = math.sqrt(I.kelvin(1e-5) / sysd.m_ion)
    for j in range(2):
        k = 0.5 * sysd.q[j] * sysd.Omega
        cov = np.mean(y[:, j] * y[:, 3 + j])
        sd = math.sqrt(sv ** 2 + (k * sx) ** 2)
        assert abs(cov - (-k * sx * sx)) < 5 * sx * sd / math.sqrt(n), j


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference (the oracle on the host cores, bounded samples of the sweep) prints one
    JSON line with the fields of the bench contract and the reference arm's own."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1",
                        "--cpu-seconds", "2"], cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["unit"] == "trajectories/s" and d["higher_is_better"] is True and d["value"] > 0
    assert d["dtype"] == "f64" and d["data"] == "synthetic"
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
