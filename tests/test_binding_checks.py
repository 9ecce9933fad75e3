"""The binding checks every tensor before its pointer crosses the C ABI (CPU only).

The library is replaced by a recorder and the device test by one that accepts CPU tensors. Then:

- every entry point is called with tensors laid out as the tests, the benchmark and smoke() lay them
  out, and must reach the library;
- each kind of wrong tensor (dtype, shape, layout, device, missing field) must be refused before it.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2509_15117_gb300 import binding as Bd  # noqa: E402


class Recorder:
    """Stands in for libionatom.so: every function returns IA_OK and records its name."""

    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        if name == "ia_error_string":
            return lambda code: b"recorded"

        def fn(*args):
            self.calls.append(name)
            return 0
        return fn


@pytest.fixture
def rec(monkeypatch):
    r = Recorder()
    monkeypatch.setattr(Bd, "_lib", r)
    monkeypatch.setattr(Bd, "_stream_ptr", lambda stream: ctypes.c_void_p(0))
    monkeypatch.setattr(Bd, "_on_device", lambda t: True)
    return r


N = 37


def ics(n=N):
    y = torch.zeros((n, 12), dtype=torch.float64)
    y0_soa, ph, sid = Bd.to_device_soa(y.numpy(), np.zeros(n), np.zeros(n, dtype=np.int32), device="cpu")
    return y0_soa, ph, sid


def test_conforming_tensors_reach_the_library(rec):
    y, p, s = ics()
    out = Bd.alloc_obs(N, device="cpu", y_final=True)
    order = torch.arange(N, dtype=torch.int64)
    Bd.ia_launch(1, y, p, s, out, order=order)
    Bd.ia_launch(1, y, p, None, Bd.alloc_obs(N, device="cpu"), kernel=Bd.IA_KERNEL_PLAIN)
    Bd.ia_launch_static(1, y, p, s, out)
    big = torch.zeros((12, 3 * N), dtype=torch.float64)
    Bd.ia_launch(1, big[:, N:2 * N], p, s, out)                           # a column slice: row stride 3N
    Bd.ia_launch(1, torch.empty((12, 0), dtype=torch.float64), torch.empty(0, dtype=torch.float64), None,
                 Bd.alloc_obs(0, device="cpu"))
    st = Bd.alloc_stats(7, device="cpu")
    Bd.ia_reduce_stats(1, out, N, s, 7, st)
    Bd.ia_reduce_stats(1, out, N, None, 7, st)
    g = Bd.Graph(1, y, p, s, out, type("S", (), {"cuda_stream": 0})(), order=order, cell_id=s, n_cells=7, stats=st)
    g.ptr = None
    Bd.ia_autotune(1, y, p, s, attempt_cap=64)
    dy0 = torch.zeros((4, 12, N), dtype=torch.float64)
    tan = Bd.alloc_tangent(N, 4, dy_final=True, device="cpu")
    Bd.ia_launch_tangent(1, y, p, s, out, dy0, np.zeros((4, 3)), tan)
    Bd.ia_launch_tangent(1, y, p, s, out, dy0[:1].contiguous(), np.zeros((1, 3)), Bd.alloc_tangent(N, 1, device="cpu"))
    Bd.ia_launch_adjoint(1, y, p, s, out, Bd.alloc_adjoint(N, 4, device="cpu"), dy0, np.zeros((4, 3)))
    Bd.ia_launch_adjoint(1, y, p, s, out, Bd.alloc_adjoint(N, 0, device="cpu"), seg=16, max_ckpt=4)
    Bd.ia_launch_adjoint(1, y, p, s, out, {})                             # the library refuses this one
    Bd.ia_launch(1, y, p, s, out, scratch=torch.zeros(4096, dtype=torch.float64))
    smp = Bd.make_sampler(Bd.IA_SAMPLE_HEAD_ON, {"m_ion": 1.0, "m_atom": 1.0, "Omega": 1.0, "q": (0.1, -0.1, 0.0),
                                                 "r0": 10.0}, seed=1, E=1.0)
    Bd.ia_sample_ics(smp, 0, y, p)
    Bd.ia_sample_ics(smp, 5, big[:, :N], p)
    Bd.ia_philox4x64(1, 2, 3, 0, torch.zeros((N, 4), dtype=torch.int64))
    Bd.ia_rcp_check(p, torch.zeros(N, dtype=torch.float64))
    Q = Bd.Queue(1, N, slice_budget=300)
    Q.launch(y, p, s, out, 5, order=order)
    Q.launch(y, p, s, out, N - 5, order=order)
    Q.state()
    Q.reset()
    assert rec.calls.count("ia_launch") == 5 and rec.calls.count("ia_launch_adjoint") == 3
    assert rec.calls.count("ia_queue_launch") == 2
    for name in ("ia_launch_static", "ia_reduce_stats", "ia_graph_create", "ia_autotune", "ia_launch_tangent",
                 "ia_sample_ics", "ia_philox4x64", "ia_rcp_check", "ia_queue_create", "ia_queue_state",
                 "ia_queue_reset"):
        assert name in rec.calls, name


def refused(fn, *args, **kw):
    with pytest.raises(Bd.IaArgumentError):
        fn(*args, **kw)


def test_wrong_tensors_are_refused_before_the_library(rec):
    y, p, s = ics()
    out = Bd.alloc_obs(N, device="cpu")
    refused(Bd.ia_launch, 1, y.t().contiguous(), p, s, out)               # (n, 12) instead of (12, n)
    refused(Bd.ia_launch, 1, y.float(), p, s, out)                         # float32
    refused(Bd.ia_launch, 1, torch.zeros((12, 2 * N), dtype=torch.float64)[:, ::2], p, s, out)  # strided columns
    refused(Bd.ia_launch, 1, y, p[:N - 1].contiguous(), s, out)           # lengths disagree
    refused(Bd.ia_launch, 1, y, p, s.long(), out)                         # sys_id int64
    refused(Bd.ia_launch, 1, y, p, s, out, order=torch.arange(N, dtype=torch.int32))
    bad = dict(out)
    bad["status"] = bad["status"].double()
    refused(Bd.ia_launch, 1, y, p, s, bad)
    bad = dict(out)
    del bad["n_rej"]
    refused(Bd.ia_launch, 1, y, p, s, bad)
    refused(Bd.ia_launch, 1, y, p, s, Bd.alloc_obs(N - 1, device="cpu"))  # outputs too short
    yf = dict(out, y_final=torch.zeros((N, 12), dtype=torch.float64))
    refused(Bd.ia_launch, 1, y, p, s, yf)
    refused(Bd.ia_reduce_stats, 1, out, N, s, 7, Bd.alloc_stats(6, device="cpu"))
    refused(Bd.ia_reduce_stats, 1, out, N, s[:3].contiguous(), 7, Bd.alloc_stats(7, device="cpu"))
    dy0 = torch.zeros((4, 12, N), dtype=torch.float64)
    refused(Bd.ia_launch_tangent, 1, y, p, s, out, dy0.transpose(1, 2), np.zeros((4, 3)),
            Bd.alloc_tangent(N, 4, device="cpu"))
    refused(Bd.ia_launch_tangent, 1, y, p, s, out, dy0, np.zeros((4, 3)), Bd.alloc_tangent(N, 3, device="cpu"))
    refused(Bd.ia_launch_tangent, 1, y, p, s, out, dy0, np.zeros((2, 3)), Bd.alloc_tangent(N, 4, device="cpu"))
    refused(Bd.ia_launch_tangent, 1, y, p, s, out, torch.zeros((5, 12, N), dtype=torch.float64), np.zeros((5, 3)),
            Bd.alloc_tangent(N, 5, device="cpu"))
    adj = Bd.alloc_adjoint(N, 0, device="cpu")
    adj["grad_y0"] = torch.zeros((4, N, 12), dtype=torch.float64)
    refused(Bd.ia_launch_adjoint, 1, y, p, s, out, adj)
    refused(Bd.ia_launch_adjoint, 1, y, p, s, out, Bd.alloc_adjoint(N, 0, device="cpu"), dy0, np.zeros((4, 3)))
    refused(Bd.ia_philox4x64, 1, 2, 3, 0, torch.zeros((N, 3), dtype=torch.int64))
    refused(Bd.ia_sample_ics, Bd.ia_sampler(), 0, y[:, :5], p)
    refused(Bd.ia_launch, 1, y, p, s, out, scratch=torch.zeros((8, 8), dtype=torch.float64).t())
    Q = Bd.Queue(1, N)
    rec.calls.clear()
    refused(Q.launch, y[:, :N - 1], p[:N - 1].contiguous(), s[:N - 1].contiguous(), out, 3)  # not the queue's n
    refused(Q.launch, y, p, s, Bd.alloc_obs(N - 1, device="cpu"), 3)
    refused(Q.launch, y.float(), p, s, out, 3)
    assert rec.calls == []


def test_host_tensors_are_refused(monkeypatch):
    monkeypatch.setattr(Bd, "_lib", Recorder())
    y, p, s = ics()
    with pytest.raises(Bd.IaArgumentError, match="CUDA device"):
        Bd.ia_launch(1, y, p, s, Bd.alloc_obs(N, device="cpu"))
