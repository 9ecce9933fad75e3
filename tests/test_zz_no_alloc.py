"""The allocation-free launch (ia_launch_static) gives the same results as ia_launch.

It is for callers that cannot allocate device memory when they launch (graph capture, host programs
that own the device memory pool, real-time loops): its scratch is a fixed array inside the library.
Collected last on purpose, so a run that stops at the first failure has run every other test first.
"""
import numpy as np
import pytest

from paper_2509_15117_gb300 import binding as Bd
from paper_2509_15117_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    Bd.load()
    return torch


def _results(out):
    return Bd.to_numpy(out)


def test_static_launch_matches_launch_twice_in_a_row(cuda):
    torch = cuda
    systems, y0, phi0, sid = I.c1_workload(24)  # 576 head-on trajectories
    descs = [s.as_dict() for s in systems]
    kw = dict(slice_budget=500)  # most trajectories pass through the suspend records (scratch)
    with Bd.System(descs) as S:
        yd, pd, sd = Bd.to_device_soa(y0, phi0, sid)
        n = len(phi0)
        ref = Bd.alloc_obs(n, y_final=True)
        Bd.ia_launch(S.handle, yd, pd, sd, ref, kernel=Bd.IA_KERNEL_PERSISTENT, **kw)
        torch.cuda.synchronize()
        ref = _results(ref)
        for call in range(2):
            out = Bd.alloc_obs(n, y_final=True)
            Bd.ia_launch_static(S.handle, yd, pd, sd, out, **kw)
            torch.cuda.synchronize()
            assert Bd.ia_static_phases(S.handle)[2] == 0, f"call {call}: a bounded wait ran out"
            got = _results(out)
            # same kernels and arithmetic: identical bits (tighter than the parity tolerance)
            for k in ref:
                np.testing.assert_array_equal(got[k], ref[k], err_msg=f"call {call}: {k}")
        assert np.mean(ref["n_steps"] + ref["n_rej"] > 500) > 0.5


def test_static_launch_rejects_sizes_beyond_its_array(cuda):
    systems, y0, phi0, sid = I.c1_workload(4)
    descs = [s.as_dict() for s in systems]
    with Bd.System(descs) as S:
        yd, pd, sd = Bd.to_device_soa(y0, phi0, sid)
        out = Bd.alloc_obs(len(phi0))
        fits = Bd.IA_STATIC_MAX_RECORDS
        assert Bd.ia_scratch_bytes(len(phi0), kernel=Bd.IA_KERNEL_PERSISTENT,
                                   suspend_capacity=fits) <= Bd.IA_STATIC_SCRATCH_BYTES
        assert Bd.ia_scratch_bytes(len(phi0), kernel=Bd.IA_KERNEL_PERSISTENT,
                                   suspend_capacity=fits + 1) > Bd.IA_STATIC_SCRATCH_BYTES
        with pytest.raises(Bd.IaError, match="size beyond"):
            Bd.ia_launch_static(S.handle, yd, pd, sd, out, suspend_capacity=fits + 1)
        # the largest capacity that fits is accepted
        Bd.ia_launch_static(S.handle, yd, pd, sd, out, suspend_capacity=fits)
        cuda.cuda.synchronize()
