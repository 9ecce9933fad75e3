"""CUDA path against the CPU oracle, through the C ABI (needs a GB300)."""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2509_15117_gb300 import binding as Bd
from paper_2509_15117_gb300 import inputs as I
from tests import parity as PY
from tests import twobody as TB

pytestmark = pytest.mark.gpu

NTHREADS = 0  # all host cores


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    Bd.load()
    return torch


def run_gpu(descs, y0, phi0, sid, kernel, y_final=False, **kw):
    with Bd.System(descs) as S:
        r = Bd.to_numpy(S.run(y0, phi0, sid, kernel=kernel, y_final=y_final, **kw))
        if kernel == Bd.IA_KERNEL_PERSISTENT:
            assert Bd.ia_launch_phases(S.handle)[2] == 0, "a bounded wait ran out"
        return r


@pytest.fixture(scope="module")
def c1(torch_cuda):
    systems, y0, phi0, sid = I.c1_workload(32)
    descs = [s.as_dict() for s in systems]
    orc, spread = PY.oracle_with_spread(descs, y0, phi0, sid, nthreads=NTHREADS)
    return descs, y0, phi0, sid, orc, spread


@pytest.mark.parametrize("kernel", [Bd.IA_KERNEL_PLAIN, Bd.IA_KERNEL_PERSISTENT])
def test_c1_per_trajectory_parity(c1, kernel):
    """Yb+-Rb head-on 32x32 octant grid (1024 trajectories, several warps and blocks), observables, bounce
    times and final states."""
    descs, y0, phi0, sid, orc, spread = c1
    g = run_gpu(descs, y0, phi0, sid, kernel, y_final=True)
    rep = PY.compare(g, orc, spread)
    print("C1 parity", kernel, rep)
    assert rep["n_single"] > 300


def test_c1_complex_lifetimes(c1):
    """Fig. 2: the lifetimes of the complexes of the head-on map (t_last - t_first bounce) have the same
    distribution on both sides, and so has each complex's number of bounces."""
    descs, y0, phi0, sid, orc, spread = c1
    g = run_gpu(descs, y0, phi0, sid, Bd.IA_KERNEL_PERSISTENT)
    rep = PY.lifetimes_agree(g, orc)
    print("C1 lifetimes", rep)
    assert rep["complexes_oracle"] > 200


def test_c1_statistics(c1):
    descs, y0, phi0, sid, orc, spread = c1
    g = run_gpu(descs, y0, phi0, sid, Bd.IA_KERNEL_PERSISTENT)
    rep = PY.statistics_agree(g, orc)
    print("C1 statistics", rep)


def test_plain_and_persistent_agree_bitwise(c1):
    """The two kernels run the same lane code, so they produce the same bits."""
    descs, y0, phi0, sid, orc, spread = c1
    a = run_gpu(descs, y0[:300], phi0[:300], sid[:300], Bd.IA_KERNEL_PLAIN, y_final=True)
    b = run_gpu(descs, y0[:300], phi0[:300], sid[:300], Bd.IA_KERNEL_PERSISTENT, y_final=True, refill=4)
    for k in a:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


@pytest.mark.parametrize("tail_group,tail_pair,tail_sms", [(6, 1, 8), (6, 1, 64), (6, 0, 8), (8, 0, 8)])
def test_tail_kernel_bitwise_equals_plain(c1, tail_group, tail_pair, tail_sms):
    """Trajectories handed to the group-mode tail after 300 attempted steps (nearly all of C1) give
    the same bits as the one-thread-per-trajectory kernel, whether a group of one warp or a pair of
    warps (on the reserved SMs) advances them: every layout evaluates the same expressions."""
    descs, y0, phi0, sid, orc, spread = c1
    a = run_gpu(descs, y0, phi0, sid, Bd.IA_KERNEL_PLAIN, y_final=True)
    b = run_gpu(descs, y0, phi0, sid, Bd.IA_KERNEL_PERSISTENT, y_final=True, slice_budget=300,
                tail_group=tail_group, tail_pair=tail_pair, tail_sms=tail_sms)
    assert np.mean(a["n_steps"] + a["n_rej"] > 300) > 0.9
    for k in a:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


def test_suspend_overflow_and_caller_scratch(c1, torch_cuda):
    """A suspend area with room for 5 trajectories (the rest finish in their lanes), in scratch the
    caller allocates, still gives the plain kernel's bits."""
    torch = torch_cuda
    descs, y0, phi0, sid, orc, spread = c1
    n = 400
    a = run_gpu(descs, y0[:n], phi0[:n], sid[:n], Bd.IA_KERNEL_PLAIN)
    kw = dict(kernel=Bd.IA_KERNEL_PERSISTENT, slice_budget=200, suspend_capacity=5)
    nbytes = Bd.ia_scratch_bytes(n, **kw)
    assert nbytes == 1024 + 256 + 5 * 256
    scratch = torch.zeros(nbytes // 8, dtype=torch.float64, device="cuda")
    assert scratch.data_ptr() % 256 == 0
    with Bd.System(descs) as S:
        yd, pd, sd = Bd.to_device_soa(y0[:n], phi0[:n], sid[:n])
        out = Bd.alloc_obs(n)
        Bd.ia_launch(S.handle, yd, pd, sd, out, scratch=scratch, **{k: v for k, v in kw.items() if k != "kernel"})
        torch.cuda.synchronize()
        b = Bd.to_numpy(out)
        ctr = scratch[:128].view(torch.int64).cpu().numpy()
    # counter layout (ia_capi.cu, checked there by a static_assert): errors at byte 16, suspend
    # records taken at byte 824
    assert ctr[824 // 8] > 5  # more trajectories asked to suspend than there was room for
    assert ctr[16 // 8] == 0  # no bounded wait ran out
    for k in a:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


def test_queue_order_and_noncooperative_fallback(c1, torch_cuda):
    """A work-queue permutation, and a grid too large for a cooperative launch (tail workers then never
    wait), change only the schedule: same bits as the plain kernel."""
    torch = torch_cuda
    descs, y0, phi0, sid, orc, spread = c1
    n = 600
    a = run_gpu(descs, y0[:n], phi0[:n], sid[:n], Bd.IA_KERNEL_PLAIN)
    perm = torch.from_numpy(np.random.default_rng(3).permutation(n).astype(np.int64)).cuda()
    with Bd.System(descs) as S:
        yd, pd, sd = Bd.to_device_soa(y0[:n], phi0[:n], sid[:n])
        for kw in ({"order": perm, "slice_budget": 400, "tail_sms": 4},
                   {"order": perm, "slice_budget": 400, "grid": 2000},
                   {"slice_budget": 400, "tail_sms": -1}):
            out = Bd.alloc_obs(n)
            Bd.ia_launch(S.handle, yd, pd, sd, out, **kw)
            torch.cuda.synchronize()
            b = Bd.to_numpy(out)
            for k in a:
                np.testing.assert_array_equal(a[k], b[k], err_msg=f"{k} {list(kw)}")


def test_rcp_newton_accuracy(torch_cuda):
    """1/r^2 from an FP32 seed refined by one third-order step stays within 2 ulp of the correctly
    rounded reciprocal over the whole range the integrator meets (and beyond, through its division
    fallback)."""
    torch = torch_cuda
    rng = np.random.default_rng(11)
    x = np.concatenate([10.0 ** rng.uniform(-40, 40, 200000), [1.0, 2.0, 3.0, 1e-300, 1e300, 5000.0 ** 2]])
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    Bd.ia_rcp_check(xd, yd)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    ref = 1.0 / x
    ulp = np.spacing(np.abs(ref))
    assert np.max(np.abs(y - ref) / ulp) <= 2.0


@pytest.mark.parametrize("n", [1, 31, 33, 129, 1025])
def test_ragged_sizes(torch_cuda, n):
    """Partial warps, partial blocks and refill tails; all trajectories written exactly once."""
    systems, y0, phi0, sid = I.c1_workload(33)
    descs = [s.as_dict() for s in systems]
    idx = np.arange(n) * 7 % len(y0)
    orc, spread = PY.oracle_with_spread(descs, y0[idx], phi0[idx], sid[idx], nthreads=NTHREADS)
    for kernel, kw in ((Bd.IA_KERNEL_PLAIN, {}), (Bd.IA_KERNEL_PERSISTENT, {"grid": 3, "block": 64}),
                       (Bd.IA_KERNEL_PERSISTENT, {"refill": 32}),
                       (Bd.IA_KERNEL_PERSISTENT, {"slice_budget": 1000, "regs_variant": 3})):
        g = run_gpu(descs, y0[idx], phi0[idx], sid[idx], kernel, **kw)
        PY.compare(g, orc, spread)


def test_mixed_systems_table(torch_cuda):
    """Five species x eight energies in one launch (sys_id per trajectory), 6x6 grid subsample each."""
    systems, y0, phi0, sid = I.c2_workload(n_grid=96, stride=16, offset=3)
    descs = [s.as_dict() for s in systems]
    orc, spread = PY.oracle_with_spread(descs, y0, phi0, sid, nthreads=NTHREADS)
    g = run_gpu(descs, y0, phi0, sid, Bd.IA_KERNEL_PERSISTENT)
    rep = PY.compare(g, orc, spread)
    print("mixed parity", rep)


def test_status_edge_cases(torch_cuda):
    systems, y0, phi0, sid = I.c1_workload(4)
    d = systems[0].as_dict()
    bad = y0[:6].copy()
    bad[0, 9] = np.nan
    bad[1, 6:9] = 0.0
    bad[2, 0] = np.inf
    sid6 = np.array([0, 0, 0, 0, 5, -1], dtype=np.int32)
    for kernel in (Bd.IA_KERNEL_PLAIN, Bd.IA_KERNEL_PERSISTENT):
        g = run_gpu([d], bad, np.zeros(6), sid6, kernel, y_final=True)
        o = O.run_batch([d], bad, np.zeros(6), sys_id=sid6)
        for k in (0, 1, 2, 4, 5):
            assert g["status"][k] == Bd.ST_BAD_IC and o["status"][k] == O.BAD_IC
            assert g["n_steps"][k] == 0 and g["theta_s"][k] == 0.0
        np.testing.assert_array_equal(g["y_final"][4], bad[4])
        assert g["status"][3] in (0, Bd.ST_COMPLEX)
    # t_max stop: same final time, status, and state at t_max to the oracle's noise
    short = dict(d)
    short["t_max"] = 1e9
    g = run_gpu([short], y0[2:3], np.zeros(1), None, Bd.IA_KERNEL_PERSISTENT, y_final=True)
    o = O.run_batch([short], y0[2:3], np.zeros(1))
    assert g["status"][0] == Bd.ST_TMAX and g["t_final"][0] == 1e9
    assert g["n_steps"][0] == o["n_steps"][0] and g["n_rej"][0] == o["n_rej"][0]
    np.testing.assert_allclose(g["y_final"][0], o["y_final"][0], rtol=1e-12, atol=1e-20)
    # attempted-step cap
    capped = dict(d)
    capped["max_attempts"] = 50
    g = run_gpu([capped], y0[2:3], np.zeros(1), None, Bd.IA_KERNEL_PLAIN)
    assert g["status"][0] == Bd.ST_MAX_STEPS and g["n_steps"][0] + g["n_rej"][0] == 50
    # empty batch is a no-op
    with Bd.System([d]) as S:
        import torch
        out = Bd.alloc_obs(0)
        Bd.ia_launch(S.handle, torch.empty((12, 0), dtype=torch.float64, device="cuda"),
                     torch.empty(0, dtype=torch.float64, device="cuda"), None, out)


def test_trap_off_kinematic_limits_gpu(torch_cuda):
    """The CUDA path converges to the two-body closed forms with the trap off (as the oracle does)."""
    errs = {}
    for rtol in (1e-10, 1e-12):
        sysd = I.make_system("Rb", De_K=1.0, q=0.0, r0=5000.0, E_K=1.5e-6, rtol=rtol)
        d = sysd.as_dict()
        E = I.kelvin(1.5e-6)
        v0 = I.speed_for_energy(E, d["m_atom"])
        y0 = I.head_on(np.array([0.3, 1.1]), np.array([0.2, 1.4]), d["r0"], v0)
        g = run_gpu([d], y0, np.zeros(2), None, Bd.IA_KERNEL_PERSISTENT)
        mi, ma = d["m_ion"], d["m_atom"]
        mu = mi * ma / (mi + ma)
        tf = TB.relative_passage(d["alpha"], d["De"], mu, d["r0"], v0, 0.0)[0]
        assert np.all(g["status"] == 0) and np.all(g["n_bounce"] == 1)
        assert np.all(np.abs(g["theta_s"] - math.pi) < 1e-11)
        # the integrator's own error against the closed forms is the oracle's, trajectory by trajectory
        orc, spread = PY.oracle_with_spread([d], y0, np.zeros(2), np.zeros(2, dtype=np.int32))
        PY.compare(g, orc, spread)
        worst = max(np.max(np.abs(g["dp"] / (2 * mu * v0) - 1)),
                    np.max(np.abs(g["dE_ion"] / (4 * ma * mi / (ma + mi) ** 2 * E) - 1)),
                    np.max(np.abs(g["t_final"] / tf - 1)))
        assert worst < 2e6 * rtol
        errs[rtol] = worst
    assert errs[1e-12] < errs[1e-10] / 20.0


def test_invalid_descriptor_and_options(torch_cuda):
    systems, y0, phi0, sid = I.c1_workload(4)
    d = systems[0].as_dict()
    bad = dict(d)
    bad["m_ion"] = -1.0
    with pytest.raises(Bd.IaError):
        Bd.System([bad])
    bad = dict(d)
    bad["rf_sign"] = 0
    with pytest.raises(Bd.IaError):
        Bd.System([bad])
    with Bd.System([d]) as S:
        y, p, s = Bd.to_device_soa(y0, phi0, sid)
        out = Bd.alloc_obs(len(phi0))
        with pytest.raises(Bd.IaError):
            Bd.ia_launch(S.handle, y, p, s, out, refill=33)
        with pytest.raises(Bd.IaError):
            Bd.ia_launch(S.handle, y, p, s, out, block=96)
        with pytest.raises(Bd.IaError):
            Bd.ia_launch(S.handle, y, p, s, out, tail_group=7)
        with pytest.raises(Bd.IaError):
            Bd.ia_launch(S.handle, y, p, s, out, regs_variant=2)
