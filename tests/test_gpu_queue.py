"""A batch integrated over several launches (ia_queue_*): through the C ABI on a GB300.

The split of a batch into parts changes only the schedule. Every trajectory's arithmetic is the one of
the plain kernel, carried across launches in lane-mode carry records or group-mode suspend records,
so the results must be bit-identical to the plain kernel's whatever the split."""
import numpy as np
import pytest

from paper_2509_15117_gb300 import binding as Bd
from paper_2509_15117_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    Bd.load()
    return torch


@pytest.fixture(scope="module")
def c1(torch_cuda):
    """Yb+-Rb head-on 32 x 32 octant grid and the plain kernel's results (with final states)."""
    systems, y0, phi0, sid = I.c1_workload(32)
    descs = [s.as_dict() for s in systems]
    with Bd.System(descs) as S:
        ref = Bd.to_numpy(S.run(y0, phi0, sid, kernel=Bd.IA_KERNEL_PLAIN, y_final=True))
    return descs, y0, phi0, sid, ref


def run_parts(torch, descs, y0, phi0, sid, counts, order=None, reuse=1, **kw):
    """Integrate the batch as parts of the given sizes (summing to n); returns the numpy results of
    each repetition (the queue is reset between repetitions) and the wait errors of every part."""
    n = len(phi0)
    assert sum(counts) == n
    results, errors = [], []
    with Bd.System(descs) as S:
        y, p, d = Bd.to_device_soa(y0, phi0, sid)
        o = None if order is None else torch.from_numpy(np.asarray(order, dtype=np.int64)).cuda()
        with Bd.Queue(S.handle, n, **kw) as Q:
            for rep in range(reuse):
                if rep:
                    Q.reset()
                out = Bd.alloc_obs(n, y_final=True)
                for k, c in enumerate(counts):
                    Q.launch(y, p, d, out, c, order=o)
                    torch.cuda.synchronize()
                    errors.append(Q.phases()[2])
                    started, parts, nn = Q.state()
                    assert (started, parts, nn) == (sum(counts[:k + 1]), k + 1, n)
                results.append(Bd.to_numpy(out))
    return results, errors


def assert_same(a, b):
    for k in a:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


@pytest.mark.parametrize("counts", [[1024], [100, 0, 300, 1, 200, 423], [16] * 64])
def test_parts_bitwise_equal_plain(c1, torch_cuda, counts):
    """Default options: the head-on trajectories at 1.5 uK run thousands to millions of attempted
    steps, so every part but the last ends with lanes busy and leaves carry records."""
    descs, y0, phi0, sid, ref = c1
    res, err = run_parts(torch_cuda, descs, y0, phi0, sid, counts)
    assert err == [0] * len(counts)
    assert_same(ref, res[0])


@pytest.mark.parametrize("tail_sms,budget", [(8, 300), (2, 1000), (-1, 300)])
def test_parts_with_group_tail_across_parts(c1, torch_cuda, tail_sms, budget):
    """A small slice budget hands nearly every trajectory to the group-mode tail; the tail workers'
    trajectories are saved at the end of each part and resumed by the next (with no reserved SMs they
    wait in the suspend records until the last part), and a queue permutation reorders the starts."""
    descs, y0, phi0, sid, ref = c1
    n = len(phi0)
    perm = np.random.default_rng(5).permutation(n)
    counts = [200, 200, 0, 300, 324]
    res, err = run_parts(torch_cuda, descs, y0, phi0, sid, counts, order=perm, reuse=2,
                         slice_budget=budget, tail_sms=tail_sms)
    assert err == [0] * (2 * len(counts))
    assert_same(ref, res[0])
    assert_same(ref, res[1])


def test_queue_argument_errors(c1, torch_cuda):
    torch = torch_cuda
    descs, y0, phi0, sid, ref = c1
    n = 64
    with Bd.System(descs) as S:
        y, p, d = Bd.to_device_soa(y0[:n], phi0[:n], sid[:n])
        out = Bd.alloc_obs(n)
        with pytest.raises(Bd.IaError):
            Bd.Queue(S.handle, n, tail_pair=1)  # the paired tail is not available to queues
        with pytest.raises(Bd.IaError):
            Bd.Queue(S.handle, 0)
        with Bd.Queue(S.handle, n) as Q:
            with pytest.raises(Bd.IaError):
                Q.launch(y, p, d, out, n + 1)  # more positions than the batch has
            Q.launch(y, p, d, out, 10)
            other = Bd.alloc_obs(n)
            with pytest.raises(Bd.IaError):
                Q.launch(y, p, d, other, 10)  # the arrays of a batch are fixed by its first part
            Q.launch(y, p, d, out, n - 10)
            with pytest.raises(Bd.IaError):
                Q.launch(y, p, d, out, 0)  # the batch is complete
            torch.cuda.synchronize()
            assert Q.phases()[2] == 0
            got = Bd.to_numpy(out)
            Q.reset()
            assert Q.state() == (0, 0, n)
    for k in got:
        np.testing.assert_array_equal(got[k], ref[k][:n], err_msg=k)
