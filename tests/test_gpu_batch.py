"""Batch statistics, CUDA-graph replay, the autotuner and mixed-parameter batches (needs a GB300)."""
import math

import numpy as np
import pytest

from paper_2509_15117_gb300 import binding as Bd
from paper_2509_15117_gb300 import inputs as I
from paper_2509_15117_gb300 import statistics as St
from tests import parity as PY

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    Bd.load()
    return torch


def _lifetime_bin_np(tau):
    bits = np.asarray(tau, dtype=np.float64).view(np.int64)
    e = ((bits >> 52) & 0x7FF) - 1023
    half = ((bits & 0xFFFFFFFFFFFFF) >= 0x6A09E667F3BCD).astype(np.int64)
    b = 2 * (e - 20) + half
    b = np.where(tau > 0, b, 0)
    return np.clip(b, 0, Bd.STATS_LIFETIME_BINS - 1)


def _bounce_bin_np(nb):
    nb = np.asarray(nb, dtype=np.int64)
    b = np.where(nb > 0, 1 + np.floor(np.log2(np.maximum(nb, 1))).astype(np.int64), 0)
    return np.clip(b, 0, Bd.STATS_BOUNCE_BINS - 1)


def test_stats_match_outputs_and_reproduce(torch_cuda):
    torch = torch_cuda
    systems, y0, phi0, sid = I.c1_workload(32)
    descs = [s.as_dict() for s in systems]
    n = len(phi0)
    cells = (np.arange(n) % 7).astype(np.int32)
    cells[5] = -1  # skipped
    with Bd.System(descs) as S:
        yd, pd, sd = Bd.to_device_soa(y0, phi0, sid)
        out = Bd.alloc_obs(n)
        Bd.ia_launch(S.handle, yd, pd, sd, out)
        cd = torch.from_numpy(cells).cuda()
        a, b = Bd.alloc_stats(7), Bd.alloc_stats(7)
        Bd.ia_reduce_stats(S.handle, out, n, cd, 7, a)
        Bd.ia_reduce_stats(S.handle, out, n, cd, 7, b)
        torch.cuda.synchronize()
        g = Bd.to_numpy(out)
        ra, rb = Bd.stats_to_numpy(a), Bd.stats_to_numpy(b)
    assert ra.tobytes() == rb.tobytes()  # bit-reproducible
    for c in range(7):
        m = cells == c
        r = ra[c]
        assert r["n"] == m.sum()
        assert r["n_complex"] == np.sum(g["n_bounce"][m] >= 2)
        assert r["attempts"] == np.sum(g["n_steps"][m].astype(np.int64) + g["n_rej"][m])
        np.testing.assert_array_equal(r["bounce_hist"],
                                      np.bincount(_bounce_bin_np(g["n_bounce"][m]), minlength=Bd.STATS_BOUNCE_BINS))
        cm = m & (g["n_bounce"] >= 2)
        tau = g["t_last_bounce"][cm] - g["t_first_bounce"][cm]
        np.testing.assert_array_equal(r["lifetime_hist"],
                                      np.bincount(_lifetime_bin_np(tau), minlength=Bd.STATS_LIFETIME_BINS))
        assert r["n_status"][Bd.STATS_EXIT_SLOT] == np.sum((g["status"][m] & 0xFF) == 0)
        for bit in range(6):
            assert r["n_status"][bit] == np.sum((g["status"][m] >> bit) & 1)
        assert r["sum_dE"] == pytest.approx(math.fsum(g["dE_ion"][m]), rel=1e-12, abs=1e-30)
        assert r["sum_dE2"] == pytest.approx(math.fsum(g["dE_ion"][m] ** 2), rel=1e-12, abs=1e-40)
        s = St.summarize(r)
        assert s["P_complex_3sigma"][0] <= s["P_complex"] <= s["P_complex_3sigma"][1]


def _c4_small():
    # 250 cells, 4..256 trajectories each; t_max of 50 us keeps the longest complexes short
    return I.c4_workload(scale=1.0 / 1024, t_max_s=50e-6)


def test_graph_replay_mixed_parameter_batch(torch_cuda):
    """All 250 cells of the D_e x q x a x species sweep in one captured graph (launch + statistics);
    two replays give the bits of a direct launch."""
    torch = torch_cuda
    systems, y0, phi0, sid = _c4_small()
    descs = [s.as_dict() for s in systems]
    n = len(phi0)
    stream = torch.cuda.Stream()
    with Bd.System(descs) as S:
        yd, pd, sd = Bd.to_device_soa(y0, phi0, sid)
        ref = Bd.alloc_obs(n)
        Bd.ia_launch(S.handle, yd, pd, sd, ref, slice_budget=2000)
        st_ref = Bd.alloc_stats(len(descs))
        Bd.ia_reduce_stats(S.handle, ref, n, sd, len(descs), st_ref)
        torch.cuda.synchronize()
        ref_np, st_ref_np = Bd.to_numpy(ref), Bd.stats_to_numpy(st_ref)
        out = Bd.alloc_obs(n)
        st = Bd.alloc_stats(len(descs))
        with torch.cuda.stream(stream):
            G = Bd.Graph(S.handle, yd, pd, sd, out, stream, cell_id=sd, n_cells=len(descs), stats=st,
                         slice_budget=2000)
            for _ in range(2):
                G.launch(stream)
                stream.synchronize()
                got = Bd.to_numpy(out)
                for k in ref_np:
                    np.testing.assert_array_equal(got[k], ref_np[k], err_msg=k)
                assert Bd.stats_to_numpy(st).tobytes() == st_ref_np.tobytes()
            G.close()
    assert st_ref_np["n"].sum() == n


def test_mixed_parameter_parity_against_oracle(torch_cuda):
    """The D_e x q x a x species sweep (250 systems in one table) against the oracle, per trajectory at
    the oracle's noise floor and statistically."""
    systems, y0, phi0, sid = I.c4_workload(scale=1.0 / 2048)
    descs = [s.as_dict() for s in systems]
    orc, spread = PY.oracle_with_spread(descs, y0, phi0, sid)
    with Bd.System(descs) as S:
        g = Bd.to_numpy(S.run(y0, phi0, sid, kernel=Bd.IA_KERNEL_PERSISTENT))
    rep = PY.compare(g, orc, spread)
    print("C4 parity", rep)
    rep2 = PY.statistics_agree(g, orc)
    print("C4 statistics", rep2)


def test_autotuner_picks_a_valid_configuration(torch_cuda):
    torch = torch_cuda
    systems, y0, phi0, sid = I.c2_workload(n_grid=64, stride=2, offset=0, t_max_s=50e-6)
    descs = [s.as_dict() for s in systems]
    with Bd.System(descs) as S:
        yd, pd, sd = Bd.to_device_soa(y0, phi0, sid)
        best, ms = Bd.ia_autotune(S.handle, yd, pd, sd, attempt_cap=512)
        assert best["block"] in (64, 128, 256) and best["regs_variant"] in (1, 3) and best["refill"] in (1, 4, 16)
        assert ms > 0.0
        m = 800
        ys, ps, ss = yd[:, :m].contiguous(), pd[:m].contiguous(), sd[:m].contiguous()
        a, b = Bd.alloc_obs(m), Bd.alloc_obs(m)
        Bd.ia_launch(S.handle, ys, ps, ss, a, kernel=Bd.IA_KERNEL_PLAIN)
        Bd.ia_launch(S.handle, ys, ps, ss, b, **best)
        torch.cuda.synchronize()
        a, b = Bd.to_numpy(a), Bd.to_numpy(b)
        for k in a:
            np.testing.assert_array_equal(a[k], b[k], err_msg=k)


def test_launch_phases_are_ordered_and_bounded(torch_cuda):
    """The device-clock phase times of a persistent launch: 0 < lane phase <= total <= event time,
    on the system's own scratch and on a caller's scratch."""
    torch = torch_cuda
    systems, y0, phi0, sid = I.c1_workload(16)
    with Bd.System([s.as_dict() for s in systems]) as S:
        y, p, d = Bd.to_device_soa(y0, phi0, sid)
        for scratch in (None, torch.zeros(Bd.ia_scratch_bytes(len(phi0)) // 8 + 32, dtype=torch.float64,
                                          device="cuda")):
            out = Bd.alloc_obs(len(phi0))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            Bd.ia_launch(S.handle, y, p, d, out, scratch=scratch)
            e1.record()
            torch.cuda.synchronize()
            lane_ms, total_ms, errors = Bd.ia_launch_phases(S.handle, scratch)
            assert 0.0 < lane_ms <= total_ms <= e0.elapsed_time(e1) * 1.05 + 0.1
            assert errors == 0
