"""The workloads use the parameters the paper prints (tests/golden/paper_parameters.json, each entry
with its passage). CPU only."""
import json
import math
import os

import pytest

from paper_2509_15117_gb300 import inputs as I

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.json")))


def test_head_on_fig1_workload():
    g = GOLDEN["head_on_fig1"]
    systems, y0, phi0, sid = I.c1_workload(4)
    s = systems[0]
    assert s.m_atom == pytest.approx(I.SPECIES[g["species"]]["mass_amu"] * I.AMU_TO_ME)
    assert s.De == pytest.approx(I.kelvin(g["De_K"])) and s.r0 == g["r0_a0"]
    v0 = math.sqrt(2 * I.kelvin(g["E_uK"] * 1e-6) / s.m_atom)
    assert all(abs(math.sqrt(sum(v * v for v in row[9:12])) / v0 - 1) < 1e-14 for row in y0)
    assert all(abs(math.sqrt(sum(x * x for x in row[6:9])) / g["r0_a0"] - 1) < 1e-14 for row in y0)


def test_thermal_runs_workload():
    g = GOLDEN["thermal_runs"]
    systems, cells = I.thermal_sweep_systems()
    assert sorted({c[2] for c in cells}) == g["De_K"]
    assert all(s.r0 == g["r0_a0"] for s in systems)
    assert I.secular_omega(0.1, 2.0) == pytest.approx(0.1 * 2.0 / 2 ** 1.5)
    import inspect
    for sampler in (I.thermal_sphere, I.thermal_disk):
        assert inspect.signature(sampler).parameters["T_ion_K"].default == pytest.approx(g["T_ion_uK"] * 1e-6)


def test_energy_scan_fig4_workload():
    g = GOLDEN["energy_scan_fig4"]
    systems, E, names = I.energy_scan_systems()
    assert len(E) == g["energies"] * len(set(names))
    assert all(s.r0 == g["r0_a0"] and s.De == pytest.approx(I.kelvin(g["De_K"])) for s in systems)
    # 1 uK of temperature is 1.5 uK of collision energy through E = (3/2) k_B T
    assert 1.5 * I.kelvin(1e-6) == pytest.approx(I.kelvin(1.5e-6))


def test_r0_rule():
    g = GOLDEN["r0_rule"]
    for sp in I.C2_SPECIES:
        for E_K in I.C2_ENERGIES_K:
            r0 = I.r0_rule(I.SPECIES[sp]["alpha"], I.kelvin(E_K))
            assert g["factor"] * 0.5 * I.SPECIES[sp]["alpha"] / r0 ** 4 < I.kelvin(E_K)
