"""Parity in the regimes of the paper's Fig. 3 and Fig. 4 runs, which differ from the head-on sweep's:
the collision-energy scan (r0 = 20,000 a0, t_max = 3 ms, energies down to 30 nK, a random rf phase) and
the deep well of the thermal runs (D_e = 100 K). Initial conditions are drawn on the device, copied
back, and integrated by the oracle from the same states (needs a GB300)."""
import numpy as np
import pytest

from paper_2509_15117_gb300 import binding as Bd
from paper_2509_15117_gb300 import inputs as I
from tests import parity as PY

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    Bd.load()
    return torch


def draw_and_run(torch, descs, samplers, n_per):
    """Device-drawn initial conditions of every cell, the GPU's results, and the states as numpy."""
    n = n_per * len(descs)
    y = torch.empty((12, n), dtype=torch.float64, device="cuda")
    ph = torch.empty((n,), dtype=torch.float64, device="cuda")
    sid = torch.arange(len(descs), dtype=torch.int32, device="cuda").repeat_interleave(n_per)
    for c, smp in enumerate(samplers):
        a = c * n_per
        Bd.ia_sample_ics(smp, a, y[:, a:a + n_per], ph[a:a + n_per])
    with Bd.System(descs) as S:
        out = Bd.alloc_obs(n, y_final=True)
        Bd.ia_launch(S.handle, y, ph, sid, out)
        torch.cuda.synchronize()
        assert Bd.ia_launch_phases(S.handle)[2] == 0
        g = Bd.to_numpy(out)
    return g, y.cpu().numpy().T.copy(), ph.cpu().numpy(), sid.cpu().numpy()


def test_energy_scan_regime(torch_cuda):
    """Fig. 4 setup: each species at 30 nK, 5.8 uK (the middle of the scan) and 1 mK, 64 head-on
    trajectories per cell with (theta, phi) uniform on the octant and a random rf phase."""
    systems, energies, names = I.energy_scan_systems()
    pick = [k for k in range(len(systems)) if k % 100 in (0, 50, 99)]
    descs = [systems[k].as_dict() for k in pick]
    samplers = [Bd.make_sampler(Bd.IA_SAMPLE_HEAD_ON, descs[c], 4004, E=float(energies[k]))
                for c, k in enumerate(pick)]
    g, y0, phi0, sid = draw_and_run(torch_cuda, descs, samplers, 64)
    assert descs[0]["r0"] == 20000.0 and abs(descs[0]["t_max"] * I.AU_TIME_S - 3e-3) < 1e-12
    orc, spread = PY.oracle_with_spread(descs, y0, phi0, sid)
    rep = PY.compare(g, orc, spread)
    print("energy-scan regime parity", rep)
    rep2 = PY.statistics_agree(g, orc)
    print("energy-scan regime statistics", rep2)
    assert rep["n_single"] > 200


def test_deep_well_regime(torch_cuda):
    """Fig. 3 setup at D_e = 100 K: Rb and Cs at 10 uK and 1 mK, 128 trajectories per cell drawn with the
    paper's sphere sampler (atom uniform on the r0 sphere, Gaussian velocity flipped inward, ion Gaussian
    at 10 uK), random rf phase."""
    systems, cells = I.thermal_sweep_systems()
    pick = [k for k, (sp, T, De) in enumerate(cells) if De == 100.0 and sp in ("Rb", "Cs") and T in (1e-5, 1e-3)]
    assert len(pick) == 4
    descs = [systems[k].as_dict() for k in pick]
    samplers = [Bd.make_sampler(Bd.IA_SAMPLE_SPHERE, descs[c], 3100, kT=I.kelvin(cells[k][1]),
                                kT_ion=I.kelvin(10e-6)) for c, k in enumerate(pick)]
    g, y0, phi0, sid = draw_and_run(torch_cuda, descs, samplers, 128)
    orc, spread = PY.oracle_with_spread(descs, y0, phi0, sid)
    rep = PY.compare(g, orc, spread)
    print("D_e = 100 K parity", rep)
    rep2 = PY.statistics_agree(g, orc)
    print("D_e = 100 K statistics", rep2)
    assert rep["n_single"] > 100
