"""Parity at full size: the whole species x energy sweep (41,943,040 trajectories) in the launch
configuration the benchmark times (persistent kernel, default options, queue order), checked against
the oracle on a seeded random sample of trajectories and, over all of them, against properties that hold
at any size (needs a GB300; about three minutes)."""
import math

import numpy as np
import pytest

import bench
from paper_2509_15117_gb300 import binding as Bd
from tests import parity as PY

pytestmark = pytest.mark.gpu

N_SAMPLE = 512


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    Bd.load()
    return torch


def test_whole_sweep_sampled_parity_and_invariants(torch_cuda):
    torch = torch_cuda
    systems, y0, phi0, sid, order = bench.step_inputs(0, 1, 0, 1)
    n = len(phi0)
    assert n == 5 * 8 * 1024 * 1024
    descs = [s.as_dict() for s in systems]
    with Bd.System(descs) as S:
        yd, pd, sd = Bd.to_device_soa(y0, phi0, sid)
        out = Bd.alloc_obs(n)
        Bd.ia_launch(S.handle, yd, pd, sd, out, order=torch.from_numpy(order).cuda())
        torch.cuda.synchronize()
        assert Bd.ia_launch_phases(S.handle)[2] == 0, "a bounded wait ran out"
        del yd, pd, sd
        g = Bd.to_numpy(out)
    # properties of every trajectory
    st = g["status"] & 0xFF
    assert not np.any(st & (Bd.ST_BAD_IC | (1 << 3) | (1 << 2) | (1 << 1))), "BAD_IC, NONFINITE, H_UNDERFLOW or MAX_STEPS"
    exits = st == 0
    assert exits.mean() > 0.99
    assert np.all(g["n_bounce"][exits] >= 1)
    assert np.all((g["theta_s"] >= 0.0) & (g["theta_s"] <= math.pi))
    assert np.all(g["dp"] >= 0.0) and np.all(g["t_final"] > 0.0)
    assert np.array_equal((g["status"] & Bd.ST_COMPLEX) != 0, g["n_bounce"] >= 2)
    assert np.all(g["n_steps"] >= 1)
    # per-trajectory parity on a seeded random sample, computed one by one by the oracle
    idx = np.sort(np.random.default_rng(20241).choice(n, N_SAMPLE, replace=False))
    orc, spread = PY.oracle_with_spread(descs, y0[idx], phi0[idx], sid[idx], nthreads=0)
    gs = {k: v[idx] for k, v in g.items()}
    rep = PY.compare(gs, orc, spread, max_flip=0.05)
    print("full-size sampled parity", rep)
    assert rep["n_single"] > N_SAMPLE // 4
