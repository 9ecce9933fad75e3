"""ia_system_create validates every descriptor before any CUDA call (CPU only): a descriptor that
passes reaches the device query (IA_ERR_NO_DEVICE on a machine without a GPU), one that fails returns
IA_ERR_BAD_DESC. Pinned here:

- the trap's Mathieu stability, against textbook values of Mathieu's characteristic curves: at
  a = 0 the first stability region ends at q = 0.908046 (the b_1 boundary). Near q = 0 its lower
  edge is a_0(q) = -q^2/2 + 7 q^4/128 - ...;
- every workload the tests, the benchmark and smoke() build is accepted.
"""
import ctypes
import math

import pytest

from paper_2509_15117_gb300 import binding as Bd
from paper_2509_15117_gb300 import inputs as I

BAD_DESC, NO_DEVICE = -2, -5


def create(descs):
    L = Bd.load()
    arr = (Bd.ia_system_desc * len(descs))(*[Bd.make_desc(d) for d in descs])
    h = ctypes.c_void_p()
    return L.ia_system_create(arr, len(descs), ctypes.byref(h))


def trap(a_xy, q_xy, a_z=None, q_z=0.0):
    d = I.make_system("Rb").as_dict()
    d["a"] = (a_xy, a_xy, -2.0 * a_xy if a_z is None else a_z)
    d["q"] = (q_xy, -q_xy, q_z)
    return d


@pytest.fixture(scope="module", autouse=True)
def no_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("checks the pre-device validation path; a GPU would create the table")


@pytest.mark.parametrize("q,ok", [(0.1, True), (0.5, True), (0.90, True), (0.92, False), (1.2, False)])
def test_stability_edge_at_a_zero(q, ok):
    assert create([trap(0.0, q)]) == (NO_DEVICE if ok else BAD_DESC)


@pytest.mark.parametrize("q", [0.05, 0.1, 0.2])
def test_lower_edge_a0(q):
    a0 = -q * q / 2 + 7 * q ** 4 / 128
    margin = 0.02 * q * q
    assert create([trap(a0 + margin, q, a_z=0.0)]) == NO_DEVICE
    assert create([trap(a0 - margin, q, a_z=0.0)]) == BAD_DESC


def test_static_axes():
    assert create([trap(0.0, 0.0)]) == NO_DEVICE                 # trap off: free ion, trace exactly 2
    assert create([trap(-0.001, 0.1)]) == NO_DEVICE              # a_z = +0.002 confines z
    assert create([trap(0.001, 0.1)]) == BAD_DESC                # a_z = -0.002 expels the ion along z
    assert create([trap(0.0, 0.1, a_z=0.0, q_z=20.0)]) == BAD_DESC  # beyond the documented range


def test_one_bad_row_rejects_the_table():
    assert create([trap(0.0, 0.1)] * 5 + [trap(0.0, 0.95)]) == BAD_DESC


def test_every_workload_is_accepted():
    tables = {
        "c1": [s.as_dict() for s in I.c1_workload(4)[0]],
        "c2": [s.as_dict() for (_, _, s) in I.c2_systems()],
        "c3": [s.as_dict() for s in I.c3_workload(4)[0]],
        "c4": [s.as_dict() for s in I.c4_workload(scale=0.001)[0]],
        "c5": [I.c5_workload(4)[0].as_dict()],
        "energy_scan": [s.as_dict() for s in I.energy_scan_systems()[0]],
        "thermal_sweep": [s.as_dict() for s in I.thermal_sweep_systems()[0]],
        "trap_off": [I.make_system("Rb", q=0.0).as_dict()],
        "li_q": [I.make_system("Li", q=q, r0=20000.0).as_dict() for q in (0.05, 0.1, 0.2, 0.3, 0.4)],
    }
    for name, descs in tables.items():
        assert create(descs) == NO_DEVICE, name
    assert len(tables["c4"]) == 250
