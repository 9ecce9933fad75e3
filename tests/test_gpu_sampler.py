"""Initial conditions drawn on the device (ia_sample_ics, ia_philox4x64) against the oracle's
sampler, through the C ABI (needs a GB300).

- The generator is integer work, so it must be bit-exact against the oracle's Philox4x64-10 and
  numpy's Philox.
- The rf phase is one IEEE product of the exact uniform, so it is bit-exact too.
- The states go through log, sqrt, sin and cos, whose last bits differ between CUDA's and the C
  library's implementations. Each component must agree within 1e-13 of its column's scale, several
  hundred times the few-ulp error of those functions.
- Trajectories integrated from device-drawn states must match the oracle's integration of the oracle's
  own draws, under the per-trajectory parity criterion of the other parity tests.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2509_15117_gb300 import binding as Bd
from paper_2509_15117_gb300 import inputs as I
from tests import parity as PY

pytestmark = pytest.mark.gpu

REL = 1e-13


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    Bd.load()
    return torch


def rb(r0=5000.0):
    return I.make_system("Rb", r0=r0).as_dict()


def draw_gpu(torch, kind, d, seed, first, n, pad=0, **kw):
    """Device draw into a (12, n + pad) buffer filled with NaN; returns (y (n, 12), phi0, untouched pad)."""
    ld = n + pad
    y = torch.full((12, ld), float("nan"), dtype=torch.float64, device="cuda")
    ph = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    Bd.ia_sample_ics(Bd.make_sampler(kind, d, seed, **kw), first, y[:, :n], ph)  # row stride ld
    torch.cuda.synchronize()
    ya = y.cpu().numpy()
    return np.ascontiguousarray(ya[:, :n].T), ph.cpu().numpy(), ya[:, n:]


def test_raw_generator_bitexact(torch_cuda):
    torch = torch_cuda
    n = 100_003
    for key0, key1, ctr1, first in ((0, 0, 0, 0), (123, 456, 7, 2 ** 40 - 17), (2 ** 64 - 1, 5, 2 ** 63, 3)):
        out = torch.empty((n, 4), dtype=torch.int64, device="cuda")
        Bd.ia_philox4x64(key0, key1, ctr1, first, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint64)
        want = O.philox4x64_stream(key0, key1, ctr1, first, n)
        np.testing.assert_array_equal(got, want)
    # and against numpy's own Philox, which advances (c0, c1, ...) by one before each block
    bg = np.random.Philox(key=np.array([123, 456], dtype=np.uint64), counter=np.array([99, 7, 0, 0], dtype=np.uint64))
    out = torch.empty((8, 4), dtype=torch.int64, device="cuda")
    Bd.ia_philox4x64(123, 456, 7, 100, out)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy().view(np.uint64).ravel(), bg.random_raw(32))


CASES = {
    "head_on": (Bd.IA_SAMPLE_HEAD_ON, dict(E=I.kelvin(1.5e-6))),
    "head_on_fixed_phase": (Bd.IA_SAMPLE_HEAD_ON, dict(E=I.kelvin(1e-5), random_phase=False, phase=1.25)),
    "sphere": (Bd.IA_SAMPLE_SPHERE, dict(kT=I.kelvin(1e-4), kT_ion=I.kelvin(1e-5))),
    "sphere_cold_ion": (Bd.IA_SAMPLE_SPHERE, dict(kT=I.kelvin(1e-6), kT_ion=0.0, micromotion=True)),
    "disk": (Bd.IA_SAMPLE_DISK, dict(kT=I.kelvin(1e-3), kT_ion=I.kelvin(1e-5), b_max=2000.0)),
    "disk_micromotion": (Bd.IA_SAMPLE_DISK, dict(kT=I.kelvin(1e-5), kT_ion=I.kelvin(1e-5), b_max=2000.0,
                                                 micromotion=True)),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_states_match_the_oracle(torch_cuda, case):
    torch = torch_cuda
    kind, kw = CASES[case]
    d = rb()
    n, first, seed = 100_003, 2 ** 33 + 5, 20250917
    yg, pg, pad = draw_gpu(torch, kind, d, seed, first, n, pad=13, **kw)
    yo, po = O.sample_ics(O.make_sampler(kind, d, seed, **kw), first, n)
    assert np.all(np.isnan(pad)), "wrote past column n - 1"
    np.testing.assert_array_equal(pg, po)
    scale = np.max(np.abs(yo), axis=0)
    err = np.abs(yg - yo)
    for c in range(12):
        assert np.all(err[:, c] <= REL * scale[c]), (case, c, float(err[:, c].max()), float(scale[c]))
    if kind == Bd.IA_SAMPLE_HEAD_ON:
        assert np.all(yg[:, :6] == 0.0)


def test_chunks_and_ranks_draw_the_same_values(torch_cuda):
    torch = torch_cuda
    d = rb()
    kw = dict(kT=I.kelvin(1e-4), kT_ion=I.kelvin(1e-5), b_max=2000.0, micromotion=True)
    whole, pw, _ = draw_gpu(torch, Bd.IA_SAMPLE_DISK, d, 9, 0, 50_000, **kw)
    for a, b in ((0, 17), (17, 32_768), (32_768, 50_000)):
        part, pp, _ = draw_gpu(torch, Bd.IA_SAMPLE_DISK, d, 9, a, b - a, **kw)
        np.testing.assert_array_equal(part, whole[a:b])
        np.testing.assert_array_equal(pp, pw[a:b])


def test_integration_of_device_drawn_states(torch_cuda):
    """Disk draws at 1 mK, integrated on the GPU from the device's states and by the oracle from its own
    states: the per-trajectory parity criterion of the other parity tests."""
    torch = torch_cuda
    vth = math.sqrt(I.kelvin(1e-3) / (I.SPECIES["Rb"]["mass_amu"] * I.AMU_TO_ME))
    d = I.make_system("Rb", r0=5000.0, v_scale=vth).as_dict()
    kw = dict(kT=I.kelvin(1e-3), kT_ion=I.kelvin(1e-5), b_max=2000.0, micromotion=True)
    n = 512
    y = torch.empty((12, n), dtype=torch.float64, device="cuda")
    ph = torch.empty((n,), dtype=torch.float64, device="cuda")
    Bd.ia_sample_ics(Bd.make_sampler(Bd.IA_SAMPLE_DISK, d, 3003, **kw), 0, y, ph)
    with Bd.System([d]) as S:
        out = Bd.alloc_obs(n)
        Bd.ia_launch(S.handle, y, ph, None, out)
        torch.cuda.synchronize()
        assert Bd.ia_launch_phases(S.handle)[2] == 0
        g = Bd.to_numpy(out)
    yo, po = O.sample_ics(O.make_sampler(O.SAMPLE_DISK, d, 3003, **kw), 0, n)
    orc, spread = PY.oracle_with_spread([d], yo, po, np.zeros(n, dtype=np.int32), nthreads=0)
    rep = PY.compare(g, orc, spread)
    print("device-drawn disk states, 1 mK", rep)
    assert rep["n_single"] > n // 2


def test_rejections_leave_buffers_untouched(torch_cuda):
    torch = torch_cuda
    d = rb()
    y = torch.zeros((12, 8), dtype=torch.float64, device="cuda")
    ph = torch.zeros((8,), dtype=torch.float64, device="cuda")
    with pytest.raises(Bd.IaError):
        Bd.ia_sample_ics(Bd.make_sampler(Bd.IA_SAMPLE_DISK, d, 1, kT=1e-9, b_max=6000.0), 0, y, ph)
    with pytest.raises(Bd.IaError):
        Bd.ia_sample_ics(Bd.make_sampler(Bd.IA_SAMPLE_HEAD_ON, d, 1, E=-1.0), 0, y, ph)
    torch.cuda.synchronize()
    assert float(y.abs().sum()) == 0.0 and float(ph.abs().sum()) == 0.0
    Bd.ia_sample_ics(Bd.make_sampler(Bd.IA_SAMPLE_HEAD_ON, d, 1, E=1e-9), 0, y[:, :0], ph[:0])
