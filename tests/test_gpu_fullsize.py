"""Parity at full size: the whole species x energy sweep (41,943,040 trajectories) in the launch
configuration the benchmark times (one work queue over the batch in queue order, integrated in as many
parts as the benchmark's default steps, with the autotuner's launch options), checked against the
oracle on a seeded random sample of trajectories and, over all of them, against properties that hold at
any size (needs a GB300; about three minutes)."""
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
    args = bench.parse([])
    systems, hy, hp, hs, order = bench.sweep_in_queue_order(1, 0)
    n = int(hp.shape[0])
    assert n == 5 * 8 * 1024 * 1024
    descs = [s.as_dict() for s in systems]
    with Bd.System(descs) as S:
        yd, pd, sd = hy.cuda(), hp.cuda(), hs.cuda()
        kw, tune = bench.lane_options(args, S.handle, yd, pd, sd, 65536, 8192)
        out = Bd.alloc_obs(n)
        bounds = bench.part_bounds(n, args.steps)
        with Bd.Queue(S.handle, n, **kw) as Q:
            for k in range(args.steps):
                Q.launch(yd, pd, sd, out, int(bounds[k + 1] - bounds[k]))
                torch.cuda.synchronize()
                assert Q.phases()[2] == 0, f"part {k}: a bounded wait ran out"
        del yd, pd, sd
        g = Bd.to_numpy(out)
    print("launch options", kw, "autotune", tune)
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
    y0 = hy.numpy()[:, idx].T.copy()
    phi0, sid = hp.numpy()[idx], hs.numpy()[idx]
    orc, spread = PY.oracle_with_spread(descs, y0, phi0, sid, nthreads=0)
    gs = {k: v[idx] for k, v in g.items()}
    rep = PY.compare(gs, orc, spread)
    print("full-size sampled parity", rep)
    assert rep["n_single"] > N_SAMPLE // 4
